// GENERATED by paper_1501_01809_gb300/codegen.py -- do not edit.
// Element-tensor contractions for affine simplices (barycentric form); see codegen.py.
#pragma once
namespace fe_gen {
template <int DIM, int P> struct Elem;
template <int DIM, int P, int Q> struct Source;
template <int DIM, int P> struct Kappa;
template <int DIM, int P> struct KappaTC;


// ---- P1 Lagrange on the triangle (3 nodes) ----
template <> struct Elem<2, 1> {
  static constexpr int ND = 3;
  static constexpr int NUP = 6;
  static constexpr int NLAM = 6;
  static constexpr int STIFF_TERMS = 6;
  // K[u] for u over the upper triangle (i <= j), row-major; Lam[k] over pairs (m <= n)
  static constexpr int STIFF_OPS = 6;  // after rewriting
  template <class Ops> __device__ __forceinline__ static void stiffness_upper(const typename Ops::T* Lam, typename Ops::T* K) {
    K[0] = Lam[0];
    K[1] = Lam[1];
    K[2] = Lam[2];
    K[3] = Lam[3];
    K[4] = Lam[4];
    K[5] = Lam[5];
  }
  template <class Ops> __device__ __forceinline__ static void helmholtz_upper(const typename Ops::T* Lam, const typename Ops::T& vol, typename Ops::T* K) {
    const typename Ops::T m0 = Ops::mulc(vol, 0.16666666666666666);
    const typename Ops::T m1 = Ops::mulc(vol, 0.08333333333333333);
    K[0] = Ops::fmac(Lam[0], 1.0, m0);
    K[1] = Ops::fmac(Lam[1], 1.0, m1);
    K[2] = Ops::fmac(Lam[2], 1.0, m1);
    K[3] = Ops::fmac(Lam[3], 1.0, m0);
    K[4] = Ops::fmac(Lam[4], 1.0, m1);
    K[5] = Ops::fmac(Lam[5], 1.0, m0);
  }
  template <class Ops> __device__ __forceinline__ static void mass_upper(const typename Ops::T& vol, typename Ops::T* K) {
    const typename Ops::T m0 = Ops::mulc(vol, 0.16666666666666666);
    const typename Ops::T m1 = Ops::mulc(vol, 0.08333333333333333);
    K[0] = m0;
    K[1] = m1;
    K[2] = m1;
    K[3] = m0;
    K[4] = m1;
    K[5] = m0;
  }
  template <class Ops, bool STIFF, bool MASS> __device__ __forceinline__ static void action_upper(const typename Ops::T* Lam, const typename Ops::T& vol, const typename Ops::T* x, typename Ops::T* y) {
    typename Ops::T k;
    if constexpr (STIFF && MASS) {
      const typename Ops::T m0 = Ops::mulc(vol, 0.16666666666666666);
      const typename Ops::T m1 = Ops::mulc(vol, 0.08333333333333333);
      { k = Ops::fmac(Lam[0], 1.0, m0); y[0] = Ops::mul(k, x[0]); }
      { k = Ops::fmac(Lam[1], 1.0, m1); y[0] = Ops::fma3(k, x[1], y[0]); y[1] = Ops::mul(k, x[0]); }
      { k = Ops::fmac(Lam[2], 1.0, m1); y[0] = Ops::fma3(k, x[2], y[0]); y[2] = Ops::mul(k, x[0]); }
      { k = Ops::fmac(Lam[3], 1.0, m0); y[1] = Ops::fma3(k, x[1], y[1]); }
      { k = Ops::fmac(Lam[4], 1.0, m1); y[1] = Ops::fma3(k, x[2], y[1]); y[2] = Ops::fma3(k, x[1], y[2]); }
      { k = Ops::fmac(Lam[5], 1.0, m0); y[2] = Ops::fma3(k, x[2], y[2]); }
    }
    else if constexpr (STIFF) {
      { k = Lam[0]; y[0] = Ops::mul(k, x[0]); }
      { k = Lam[1]; y[0] = Ops::fma3(k, x[1], y[0]); y[1] = Ops::mul(k, x[0]); }
      { k = Lam[2]; y[0] = Ops::fma3(k, x[2], y[0]); y[2] = Ops::mul(k, x[0]); }
      { k = Lam[3]; y[1] = Ops::fma3(k, x[1], y[1]); }
      { k = Lam[4]; y[1] = Ops::fma3(k, x[2], y[1]); y[2] = Ops::fma3(k, x[1], y[2]); }
      { k = Lam[5]; y[2] = Ops::fma3(k, x[2], y[2]); }
    }
    else if constexpr (MASS) {
      const typename Ops::T m0 = Ops::mulc(vol, 0.16666666666666666);
      const typename Ops::T m1 = Ops::mulc(vol, 0.08333333333333333);
      { k = m0; y[0] = Ops::mul(k, x[0]); }
      { k = m1; y[0] = Ops::fma3(k, x[1], y[0]); y[1] = Ops::mul(k, x[0]); }
      { k = m1; y[0] = Ops::fma3(k, x[2], y[0]); y[2] = Ops::mul(k, x[0]); }
      { k = m0; y[1] = Ops::fma3(k, x[1], y[1]); }
      { k = m1; y[1] = Ops::fma3(k, x[2], y[1]); y[2] = Ops::fma3(k, x[1], y[2]); }
      { k = m0; y[2] = Ops::fma3(k, x[2], y[2]); }
    }
  }
  __host__ __device__ static constexpr int upper_index(int i, int j) {
    return i <= j ? i * 3 - (i * (i - 1)) / 2 + (j - i) : j * 3 - (j * (j - 1)) / 2 + (i - j);
  }
};

// ---- P2 Lagrange on the triangle (6 nodes) ----
template <> struct Elem<2, 2> {
  static constexpr int ND = 6;
  static constexpr int NUP = 21;
  static constexpr int NLAM = 6;
  static constexpr int STIFF_TERMS = 33;
  // K[u] for u over the upper triangle (i <= j), row-major; Lam[k] over pairs (m <= n)
  static constexpr int STIFF_OPS = 30;  // after rewriting
  template <class Ops> __device__ __forceinline__ static void stiffness_upper(const typename Ops::T* Lam, typename Ops::T* K) {
    const typename Ops::T w0 = Ops::add(Lam[0], Lam[1]);
    const typename Ops::T w1 = Ops::add(Lam[2], Lam[5]);
    const typename Ops::T w2 = Ops::add(Lam[3], Lam[4]);
    K[0] = Lam[0];
    K[1] = Ops::mulc(Lam[1], -0.3333333333333333);
    K[2] = Ops::mulc(Lam[2], -0.3333333333333333);
    K[3] = Ops::mulc(Lam[1], 1.3333333333333333);
    K[4] = Ops::mulc(Lam[2], 1.3333333333333333);
    K[5] = Ops::zero();
    K[6] = Lam[3];
    K[7] = Ops::mulc(Lam[4], -0.3333333333333333);
    K[8] = Ops::mulc(Lam[1], 1.3333333333333333);
    K[9] = Ops::zero();
    K[10] = Ops::mulc(Lam[4], 1.3333333333333333);
    K[11] = Lam[5];
    K[12] = Ops::zero();
    K[13] = Ops::mulc(Lam[2], 1.3333333333333333);
    K[14] = Ops::mulc(Lam[4], 1.3333333333333333);
    K[15] = Ops::fmac(w0, 2.6666666666666665, Ops::mulc(Lam[3], 2.6666666666666665));
    K[16] = Ops::fmac(w0, 1.3333333333333333, Ops::fmac(Lam[4], 2.6666666666666665, Ops::mulc(Lam[2], 1.3333333333333333)));
    K[17] = Ops::fmac(w2, 1.3333333333333333, Ops::fmac(Lam[2], 2.6666666666666665, Ops::mulc(Lam[1], 1.3333333333333333)));
    K[18] = Ops::fmac(w1, 2.6666666666666665, Ops::mulc(Lam[0], 2.6666666666666665));
    K[19] = Ops::fmac(w1, 1.3333333333333333, Ops::fmac(Lam[4], 1.3333333333333333, Ops::mulc(Lam[1], 2.6666666666666665)));
    K[20] = Ops::fmac(w2, 2.6666666666666665, Ops::mulc(Lam[5], 2.6666666666666665));
  }
  template <class Ops> __device__ __forceinline__ static void helmholtz_upper(const typename Ops::T* Lam, const typename Ops::T& vol, typename Ops::T* K) {
    const typename Ops::T w0 = Ops::add(Lam[0], Lam[1]);
    const typename Ops::T w1 = Ops::add(Lam[2], Lam[5]);
    const typename Ops::T w2 = Ops::add(Lam[3], Lam[4]);
    const typename Ops::T m0 = Ops::mulc(vol, 0.03333333333333333);
    const typename Ops::T m1 = Ops::mulc(vol, -0.005555555555555556);
    const typename Ops::T m2 = Ops::mulc(vol, -0.022222222222222223);
    const typename Ops::T m3 = Ops::mulc(vol, 0.17777777777777778);
    const typename Ops::T m4 = Ops::mulc(vol, 0.08888888888888889);
    K[0] = Ops::fmac(Lam[0], 1.0, m0);
    K[1] = Ops::fmac(Lam[1], -0.3333333333333333, m1);
    K[2] = Ops::fmac(Lam[2], -0.3333333333333333, m1);
    K[3] = Ops::mulc(Lam[1], 1.3333333333333333);
    K[4] = Ops::mulc(Lam[2], 1.3333333333333333);
    K[5] = m2;
    K[6] = Ops::fmac(Lam[3], 1.0, m0);
    K[7] = Ops::fmac(Lam[4], -0.3333333333333333, m1);
    K[8] = Ops::mulc(Lam[1], 1.3333333333333333);
    K[9] = m2;
    K[10] = Ops::mulc(Lam[4], 1.3333333333333333);
    K[11] = Ops::fmac(Lam[5], 1.0, m0);
    K[12] = m2;
    K[13] = Ops::mulc(Lam[2], 1.3333333333333333);
    K[14] = Ops::mulc(Lam[4], 1.3333333333333333);
    K[15] = Ops::fmac(w0, 2.6666666666666665, Ops::fmac(Lam[3], 2.6666666666666665, m3));
    K[16] = Ops::fmac(w0, 1.3333333333333333, Ops::fmac(Lam[4], 2.6666666666666665, Ops::fmac(Lam[2], 1.3333333333333333, m4)));
    K[17] = Ops::fmac(w2, 1.3333333333333333, Ops::fmac(Lam[2], 2.6666666666666665, Ops::fmac(Lam[1], 1.3333333333333333, m4)));
    K[18] = Ops::fmac(w1, 2.6666666666666665, Ops::fmac(Lam[0], 2.6666666666666665, m3));
    K[19] = Ops::fmac(w1, 1.3333333333333333, Ops::fmac(Lam[4], 1.3333333333333333, Ops::fmac(Lam[1], 2.6666666666666665, m4)));
    K[20] = Ops::fmac(w2, 2.6666666666666665, Ops::fmac(Lam[5], 2.6666666666666665, m3));
  }
  template <class Ops> __device__ __forceinline__ static void mass_upper(const typename Ops::T& vol, typename Ops::T* K) {
    const typename Ops::T m0 = Ops::mulc(vol, 0.03333333333333333);
    const typename Ops::T m1 = Ops::mulc(vol, -0.005555555555555556);
    const typename Ops::T m2 = Ops::mulc(vol, -0.022222222222222223);
    const typename Ops::T m3 = Ops::mulc(vol, 0.17777777777777778);
    const typename Ops::T m4 = Ops::mulc(vol, 0.08888888888888889);
    K[0] = m0;
    K[1] = m1;
    K[2] = m1;
    K[3] = Ops::zero();
    K[4] = Ops::zero();
    K[5] = m2;
    K[6] = m0;
    K[7] = m1;
    K[8] = Ops::zero();
    K[9] = m2;
    K[10] = Ops::zero();
    K[11] = m0;
    K[12] = m2;
    K[13] = Ops::zero();
    K[14] = Ops::zero();
    K[15] = m3;
    K[16] = m4;
    K[17] = m4;
    K[18] = m3;
    K[19] = m4;
    K[20] = m3;
  }
  template <class Ops, bool STIFF, bool MASS> __device__ __forceinline__ static void action_upper(const typename Ops::T* Lam, const typename Ops::T& vol, const typename Ops::T* x, typename Ops::T* y) {
    typename Ops::T k;
    if constexpr (STIFF && MASS) {
      const typename Ops::T w0 = Ops::add(Lam[0], Lam[1]);
      const typename Ops::T w1 = Ops::add(Lam[2], Lam[5]);
      const typename Ops::T w2 = Ops::add(Lam[3], Lam[4]);
      const typename Ops::T m0 = Ops::mulc(vol, 0.03333333333333333);
      const typename Ops::T m1 = Ops::mulc(vol, -0.005555555555555556);
      const typename Ops::T m2 = Ops::mulc(vol, -0.022222222222222223);
      const typename Ops::T m3 = Ops::mulc(vol, 0.17777777777777778);
      const typename Ops::T m4 = Ops::mulc(vol, 0.08888888888888889);
      { k = Ops::fmac(Lam[0], 1.0, m0); y[0] = Ops::mul(k, x[0]); }
      { k = Ops::fmac(Lam[1], -0.3333333333333333, m1); y[0] = Ops::fma3(k, x[1], y[0]); y[1] = Ops::mul(k, x[0]); }
      { k = Ops::fmac(Lam[2], -0.3333333333333333, m1); y[0] = Ops::fma3(k, x[2], y[0]); y[2] = Ops::mul(k, x[0]); }
      { k = Ops::mulc(Lam[1], 1.3333333333333333); y[0] = Ops::fma3(k, x[3], y[0]); y[3] = Ops::mul(k, x[0]); }
      { k = Ops::mulc(Lam[2], 1.3333333333333333); y[0] = Ops::fma3(k, x[4], y[0]); y[4] = Ops::mul(k, x[0]); }
      { k = m2; y[0] = Ops::fma3(k, x[5], y[0]); y[5] = Ops::mul(k, x[0]); }
      { k = Ops::fmac(Lam[3], 1.0, m0); y[1] = Ops::fma3(k, x[1], y[1]); }
      { k = Ops::fmac(Lam[4], -0.3333333333333333, m1); y[1] = Ops::fma3(k, x[2], y[1]); y[2] = Ops::fma3(k, x[1], y[2]); }
      { k = Ops::mulc(Lam[1], 1.3333333333333333); y[1] = Ops::fma3(k, x[3], y[1]); y[3] = Ops::fma3(k, x[1], y[3]); }
      { k = m2; y[1] = Ops::fma3(k, x[4], y[1]); y[4] = Ops::fma3(k, x[1], y[4]); }
      { k = Ops::mulc(Lam[4], 1.3333333333333333); y[1] = Ops::fma3(k, x[5], y[1]); y[5] = Ops::fma3(k, x[1], y[5]); }
      { k = Ops::fmac(Lam[5], 1.0, m0); y[2] = Ops::fma3(k, x[2], y[2]); }
      { k = m2; y[2] = Ops::fma3(k, x[3], y[2]); y[3] = Ops::fma3(k, x[2], y[3]); }
      { k = Ops::mulc(Lam[2], 1.3333333333333333); y[2] = Ops::fma3(k, x[4], y[2]); y[4] = Ops::fma3(k, x[2], y[4]); }
      { k = Ops::mulc(Lam[4], 1.3333333333333333); y[2] = Ops::fma3(k, x[5], y[2]); y[5] = Ops::fma3(k, x[2], y[5]); }
      { k = Ops::fmac(w0, 2.6666666666666665, Ops::fmac(Lam[3], 2.6666666666666665, m3)); y[3] = Ops::fma3(k, x[3], y[3]); }
      { k = Ops::fmac(w0, 1.3333333333333333, Ops::fmac(Lam[4], 2.6666666666666665, Ops::fmac(Lam[2], 1.3333333333333333, m4))); y[3] = Ops::fma3(k, x[4], y[3]); y[4] = Ops::fma3(k, x[3], y[4]); }
      { k = Ops::fmac(w2, 1.3333333333333333, Ops::fmac(Lam[2], 2.6666666666666665, Ops::fmac(Lam[1], 1.3333333333333333, m4))); y[3] = Ops::fma3(k, x[5], y[3]); y[5] = Ops::fma3(k, x[3], y[5]); }
      { k = Ops::fmac(w1, 2.6666666666666665, Ops::fmac(Lam[0], 2.6666666666666665, m3)); y[4] = Ops::fma3(k, x[4], y[4]); }
      { k = Ops::fmac(w1, 1.3333333333333333, Ops::fmac(Lam[4], 1.3333333333333333, Ops::fmac(Lam[1], 2.6666666666666665, m4))); y[4] = Ops::fma3(k, x[5], y[4]); y[5] = Ops::fma3(k, x[4], y[5]); }
      { k = Ops::fmac(w2, 2.6666666666666665, Ops::fmac(Lam[5], 2.6666666666666665, m3)); y[5] = Ops::fma3(k, x[5], y[5]); }
    }
    else if constexpr (STIFF) {
      const typename Ops::T w0 = Ops::add(Lam[0], Lam[1]);
      const typename Ops::T w1 = Ops::add(Lam[2], Lam[5]);
      const typename Ops::T w2 = Ops::add(Lam[3], Lam[4]);
      { k = Lam[0]; y[0] = Ops::mul(k, x[0]); }
      { k = Ops::mulc(Lam[1], -0.3333333333333333); y[0] = Ops::fma3(k, x[1], y[0]); y[1] = Ops::mul(k, x[0]); }
      { k = Ops::mulc(Lam[2], -0.3333333333333333); y[0] = Ops::fma3(k, x[2], y[0]); y[2] = Ops::mul(k, x[0]); }
      { k = Ops::mulc(Lam[1], 1.3333333333333333); y[0] = Ops::fma3(k, x[3], y[0]); y[3] = Ops::mul(k, x[0]); }
      { k = Ops::mulc(Lam[2], 1.3333333333333333); y[0] = Ops::fma3(k, x[4], y[0]); y[4] = Ops::mul(k, x[0]); }
      { k = Lam[3]; y[1] = Ops::fma3(k, x[1], y[1]); }
      { k = Ops::mulc(Lam[4], -0.3333333333333333); y[1] = Ops::fma3(k, x[2], y[1]); y[2] = Ops::fma3(k, x[1], y[2]); }
      { k = Ops::mulc(Lam[1], 1.3333333333333333); y[1] = Ops::fma3(k, x[3], y[1]); y[3] = Ops::fma3(k, x[1], y[3]); }
      { k = Ops::mulc(Lam[4], 1.3333333333333333); y[1] = Ops::fma3(k, x[5], y[1]); y[5] = Ops::mul(k, x[1]); }
      { k = Lam[5]; y[2] = Ops::fma3(k, x[2], y[2]); }
      { k = Ops::mulc(Lam[2], 1.3333333333333333); y[2] = Ops::fma3(k, x[4], y[2]); y[4] = Ops::fma3(k, x[2], y[4]); }
      { k = Ops::mulc(Lam[4], 1.3333333333333333); y[2] = Ops::fma3(k, x[5], y[2]); y[5] = Ops::fma3(k, x[2], y[5]); }
      { k = Ops::fmac(w0, 2.6666666666666665, Ops::mulc(Lam[3], 2.6666666666666665)); y[3] = Ops::fma3(k, x[3], y[3]); }
      { k = Ops::fmac(w0, 1.3333333333333333, Ops::fmac(Lam[4], 2.6666666666666665, Ops::mulc(Lam[2], 1.3333333333333333))); y[3] = Ops::fma3(k, x[4], y[3]); y[4] = Ops::fma3(k, x[3], y[4]); }
      { k = Ops::fmac(w2, 1.3333333333333333, Ops::fmac(Lam[2], 2.6666666666666665, Ops::mulc(Lam[1], 1.3333333333333333))); y[3] = Ops::fma3(k, x[5], y[3]); y[5] = Ops::fma3(k, x[3], y[5]); }
      { k = Ops::fmac(w1, 2.6666666666666665, Ops::mulc(Lam[0], 2.6666666666666665)); y[4] = Ops::fma3(k, x[4], y[4]); }
      { k = Ops::fmac(w1, 1.3333333333333333, Ops::fmac(Lam[4], 1.3333333333333333, Ops::mulc(Lam[1], 2.6666666666666665))); y[4] = Ops::fma3(k, x[5], y[4]); y[5] = Ops::fma3(k, x[4], y[5]); }
      { k = Ops::fmac(w2, 2.6666666666666665, Ops::mulc(Lam[5], 2.6666666666666665)); y[5] = Ops::fma3(k, x[5], y[5]); }
    }
    else if constexpr (MASS) {
      const typename Ops::T m0 = Ops::mulc(vol, 0.03333333333333333);
      const typename Ops::T m1 = Ops::mulc(vol, -0.005555555555555556);
      const typename Ops::T m2 = Ops::mulc(vol, -0.022222222222222223);
      const typename Ops::T m3 = Ops::mulc(vol, 0.17777777777777778);
      const typename Ops::T m4 = Ops::mulc(vol, 0.08888888888888889);
      { k = m0; y[0] = Ops::mul(k, x[0]); }
      { k = m1; y[0] = Ops::fma3(k, x[1], y[0]); y[1] = Ops::mul(k, x[0]); }
      { k = m1; y[0] = Ops::fma3(k, x[2], y[0]); y[2] = Ops::mul(k, x[0]); }
      { k = m2; y[0] = Ops::fma3(k, x[5], y[0]); y[5] = Ops::mul(k, x[0]); }
      { k = m0; y[1] = Ops::fma3(k, x[1], y[1]); }
      { k = m1; y[1] = Ops::fma3(k, x[2], y[1]); y[2] = Ops::fma3(k, x[1], y[2]); }
      { k = m2; y[1] = Ops::fma3(k, x[4], y[1]); y[4] = Ops::mul(k, x[1]); }
      { k = m0; y[2] = Ops::fma3(k, x[2], y[2]); }
      { k = m2; y[2] = Ops::fma3(k, x[3], y[2]); y[3] = Ops::mul(k, x[2]); }
      { k = m3; y[3] = Ops::fma3(k, x[3], y[3]); }
      { k = m4; y[3] = Ops::fma3(k, x[4], y[3]); y[4] = Ops::fma3(k, x[3], y[4]); }
      { k = m4; y[3] = Ops::fma3(k, x[5], y[3]); y[5] = Ops::fma3(k, x[3], y[5]); }
      { k = m3; y[4] = Ops::fma3(k, x[4], y[4]); }
      { k = m4; y[4] = Ops::fma3(k, x[5], y[4]); y[5] = Ops::fma3(k, x[4], y[5]); }
      { k = m3; y[5] = Ops::fma3(k, x[5], y[5]); }
    }
  }
  __host__ __device__ static constexpr int upper_index(int i, int j) {
    return i <= j ? i * 6 - (i * (i - 1)) / 2 + (j - i) : j * 6 - (j * (j - 1)) / 2 + (i - j);
  }
};

// ---- P3 Lagrange on the triangle (10 nodes) ----
template <> struct Elem<2, 3> {
  static constexpr int ND = 10;
  static constexpr int NUP = 55;
  static constexpr int NLAM = 6;
  static constexpr int STIFF_TERMS = 156;
  // K[u] for u over the upper triangle (i <= j), row-major; Lam[k] over pairs (m <= n)
  static constexpr int STIFF_OPS = 87;  // after rewriting
  template <class Ops> __device__ __forceinline__ static void stiffness_upper(const typename Ops::T* Lam, typename Ops::T* K) {
    const typename Ops::T w0 = Ops::add(Lam[0], Lam[1]);
    const typename Ops::T w1 = Ops::add(Lam[2], Lam[4]);
    const typename Ops::T w2 = Ops::add(Lam[1], Lam[4]);
    const typename Ops::T w3 = Ops::add(Lam[5], w1);
    const typename Ops::T w4 = Ops::add(Lam[2], w0);
    const typename Ops::T w5 = Ops::add(Lam[3], w2);
    const typename Ops::T w6 = Ops::fmac(w3, 0.5, Lam[1]);
    const typename Ops::T w7 = Ops::fmac(w5, 0.5, Lam[2]);
    const typename Ops::T w8 = Ops::fmac(w4, 0.5, Lam[4]);
    const typename Ops::T w9 = Ops::add(Lam[0], Lam[5]);
    const typename Ops::T w10 = Ops::add(Lam[3], Lam[5]);
    const typename Ops::T w11 = Ops::add(Lam[3], w0);
    const typename Ops::T w12 = Ops::add(Lam[1], Lam[2]);
    const typename Ops::T w13 = Ops::add(Lam[2], w9);
    const typename Ops::T w14 = Ops::add(Lam[4], w10);
    K[0] = Ops::mulc(Lam[0], 0.85);
    K[1] = Ops::mulc(Lam[1], 0.175);
    K[2] = Ops::mulc(Lam[2], 0.175);
    K[3] = Ops::fmac(Lam[1], 1.425, Ops::mulc(Lam[0], 0.075));
    K[4] = Ops::fmac(Lam[1], -0.6, Ops::mulc(Lam[0], 0.075));
    K[5] = Ops::fmac(Lam[2], 1.425, Ops::mulc(Lam[0], 0.075));
    K[6] = Ops::fmac(Lam[2], -0.6, Ops::mulc(Lam[0], 0.075));
    K[7] = Ops::mulc(w12, 0.075);
    K[8] = Ops::mulc(w12, 0.075);
    K[9] = Ops::mulc(w4, 0.225);
    K[10] = Ops::mulc(Lam[3], 0.85);
    K[11] = Ops::mulc(Lam[4], 0.175);
    K[12] = Ops::fmac(Lam[3], 0.075, Ops::mulc(Lam[1], -0.6));
    K[13] = Ops::fmac(Lam[3], 0.075, Ops::mulc(Lam[1], 1.425));
    K[14] = Ops::mulc(w2, 0.075);
    K[15] = Ops::mulc(w2, 0.075);
    K[16] = Ops::fmac(Lam[4], 1.425, Ops::mulc(Lam[3], 0.075));
    K[17] = Ops::fmac(Lam[4], -0.6, Ops::mulc(Lam[3], 0.075));
    K[18] = Ops::mulc(w5, 0.225);
    K[19] = Ops::mulc(Lam[5], 0.85);
    K[20] = Ops::mulc(w1, 0.075);
    K[21] = Ops::mulc(w1, 0.075);
    K[22] = Ops::fmac(Lam[5], 0.075, Ops::mulc(Lam[2], -0.6));
    K[23] = Ops::fmac(Lam[5], 0.075, Ops::mulc(Lam[2], 1.425));
    K[24] = Ops::fmac(Lam[5], 0.075, Ops::mulc(Lam[4], -0.6));
    K[25] = Ops::fmac(Lam[5], 0.075, Ops::mulc(Lam[4], 1.425));
    K[26] = Ops::mulc(w3, 0.225);
    K[27] = Ops::mulc(w11, 3.375);
    K[28] = Ops::fmac(Lam[3], -0.675, Ops::fmac(Lam[1], 1.35, Ops::mulc(Lam[0], -0.675)));
    K[29] = Ops::mulc(w8, 3.375);
    K[30] = Ops::mulc(w8, -0.675);
    K[31] = Ops::mulc(w7, -0.675);
    K[32] = Ops::mulc(w7, -0.675);
    K[33] = Ops::mulc(w7, 4.05);
    K[34] = Ops::mulc(w11, 3.375);
    K[35] = Ops::mulc(w8, -0.675);
    K[36] = Ops::mulc(w8, -0.675);
    K[37] = Ops::mulc(w7, 3.375);
    K[38] = Ops::mulc(w7, -0.675);
    K[39] = Ops::mulc(w8, 4.05);
    K[40] = Ops::mulc(w13, 3.375);
    K[41] = Ops::fmac(w9, -0.675, Ops::mulc(Lam[2], 1.35));
    K[42] = Ops::mulc(w6, -0.675);
    K[43] = Ops::mulc(w6, -0.675);
    K[44] = Ops::mulc(w6, 4.05);
    K[45] = Ops::mulc(w13, 3.375);
    K[46] = Ops::mulc(w6, -0.675);
    K[47] = Ops::mulc(w6, 3.375);
    K[48] = Ops::mulc(w8, 4.05);
    K[49] = Ops::mulc(w14, 3.375);
    K[50] = Ops::fmac(w10, -0.675, Ops::mulc(Lam[4], 1.35));
    K[51] = Ops::mulc(w6, 4.05);
    K[52] = Ops::mulc(w14, 3.375);
    K[53] = Ops::mulc(w7, 4.05);
    K[54] = Ops::fmac(w11, 8.1, Ops::mulc(w3, 8.1));
  }
  template <class Ops> __device__ __forceinline__ static void helmholtz_upper(const typename Ops::T* Lam, const typename Ops::T& vol, typename Ops::T* K) {
    const typename Ops::T w0 = Ops::add(Lam[0], Lam[1]);
    const typename Ops::T w1 = Ops::add(Lam[2], Lam[4]);
    const typename Ops::T w2 = Ops::add(Lam[1], Lam[4]);
    const typename Ops::T w3 = Ops::add(Lam[5], w1);
    const typename Ops::T w4 = Ops::add(Lam[2], w0);
    const typename Ops::T w5 = Ops::add(Lam[3], w2);
    const typename Ops::T w6 = Ops::fmac(w3, 0.5, Lam[1]);
    const typename Ops::T w7 = Ops::fmac(w5, 0.5, Lam[2]);
    const typename Ops::T w8 = Ops::fmac(w4, 0.5, Lam[4]);
    const typename Ops::T w9 = Ops::add(Lam[0], Lam[5]);
    const typename Ops::T w10 = Ops::add(Lam[3], Lam[5]);
    const typename Ops::T w11 = Ops::add(Lam[3], w0);
    const typename Ops::T w12 = Ops::add(Lam[1], Lam[2]);
    const typename Ops::T w13 = Ops::add(Lam[2], w9);
    const typename Ops::T w14 = Ops::add(Lam[4], w10);
    const typename Ops::T m0 = Ops::mulc(vol, 0.01130952380952381);
    const typename Ops::T m1 = Ops::mulc(vol, 0.001636904761904762);
    const typename Ops::T m2 = Ops::mulc(vol, 0.0026785714285714286);
    const typename Ops::T m3 = Ops::mulc(vol, 0.0040178571428571425);
    const typename Ops::T m4 = Ops::mulc(vol, 0.005357142857142857);
    const typename Ops::T m5 = Ops::mulc(vol, 0.08035714285714286);
    const typename Ops::T m6 = Ops::mulc(vol, -0.028125);
    const typename Ops::T m7 = Ops::mulc(vol, 0.04017857142857143);
    const typename Ops::T m8 = Ops::mulc(vol, -0.020089285714285716);
    const typename Ops::T m9 = Ops::mulc(vol, -0.008035714285714285);
    const typename Ops::T m10 = Ops::mulc(vol, 0.024107142857142858);
    const typename Ops::T m11 = Ops::mulc(vol, 0.2892857142857143);
    K[0] = Ops::fmac(Lam[0], 0.85, m0);
    K[1] = Ops::fmac(Lam[1], 0.175, m1);
    K[2] = Ops::fmac(Lam[2], 0.175, m1);
    K[3] = Ops::fmac(Lam[1], 1.425, Ops::fmac(Lam[0], 0.075, m2));
    K[4] = Ops::fmac(Lam[1], -0.6, Ops::mulc(Lam[0], 0.075));
    K[5] = Ops::fmac(Lam[2], 1.425, Ops::fmac(Lam[0], 0.075, m2));
    K[6] = Ops::fmac(Lam[2], -0.6, Ops::mulc(Lam[0], 0.075));
    K[7] = Ops::fmac(w12, 0.075, m3);
    K[8] = Ops::fmac(w12, 0.075, m3);
    K[9] = Ops::fmac(w4, 0.225, m4);
    K[10] = Ops::fmac(Lam[3], 0.85, m0);
    K[11] = Ops::fmac(Lam[4], 0.175, m1);
    K[12] = Ops::fmac(Lam[3], 0.075, Ops::mulc(Lam[1], -0.6));
    K[13] = Ops::fmac(Lam[3], 0.075, Ops::fmac(Lam[1], 1.425, m2));
    K[14] = Ops::fmac(w2, 0.075, m3);
    K[15] = Ops::fmac(w2, 0.075, m3);
    K[16] = Ops::fmac(Lam[4], 1.425, Ops::fmac(Lam[3], 0.075, m2));
    K[17] = Ops::fmac(Lam[4], -0.6, Ops::mulc(Lam[3], 0.075));
    K[18] = Ops::fmac(w5, 0.225, m4);
    K[19] = Ops::fmac(Lam[5], 0.85, m0);
    K[20] = Ops::fmac(w1, 0.075, m3);
    K[21] = Ops::fmac(w1, 0.075, m3);
    K[22] = Ops::fmac(Lam[5], 0.075, Ops::mulc(Lam[2], -0.6));
    K[23] = Ops::fmac(Lam[5], 0.075, Ops::fmac(Lam[2], 1.425, m2));
    K[24] = Ops::fmac(Lam[5], 0.075, Ops::mulc(Lam[4], -0.6));
    K[25] = Ops::fmac(Lam[5], 0.075, Ops::fmac(Lam[4], 1.425, m2));
    K[26] = Ops::fmac(w3, 0.225, m4);
    K[27] = Ops::fmac(w11, 3.375, m5);
    K[28] = Ops::fmac(Lam[3], -0.675, Ops::fmac(Lam[1], 1.35, Ops::fmac(Lam[0], -0.675, m6)));
    K[29] = Ops::fmac(w8, 3.375, m7);
    K[30] = Ops::fmac(w8, -0.675, m8);
    K[31] = Ops::fmac(w7, -0.675, m8);
    K[32] = Ops::fmac(w7, -0.675, m9);
    K[33] = Ops::fmac(w7, 4.05, m10);
    K[34] = Ops::fmac(w11, 3.375, m5);
    K[35] = Ops::fmac(w8, -0.675, m8);
    K[36] = Ops::fmac(w8, -0.675, m9);
    K[37] = Ops::fmac(w7, 3.375, m7);
    K[38] = Ops::fmac(w7, -0.675, m8);
    K[39] = Ops::fmac(w8, 4.05, m10);
    K[40] = Ops::fmac(w13, 3.375, m5);
    K[41] = Ops::fmac(w9, -0.675, Ops::fmac(Lam[2], 1.35, m6));
    K[42] = Ops::fmac(w6, -0.675, m9);
    K[43] = Ops::fmac(w6, -0.675, m8);
    K[44] = Ops::fmac(w6, 4.05, m10);
    K[45] = Ops::fmac(w13, 3.375, m5);
    K[46] = Ops::fmac(w6, -0.675, m8);
    K[47] = Ops::fmac(w6, 3.375, m7);
    K[48] = Ops::fmac(w8, 4.05, m10);
    K[49] = Ops::fmac(w14, 3.375, m5);
    K[50] = Ops::fmac(w10, -0.675, Ops::fmac(Lam[4], 1.35, m6));
    K[51] = Ops::fmac(w6, 4.05, m10);
    K[52] = Ops::fmac(w14, 3.375, m5);
    K[53] = Ops::fmac(w7, 4.05, m10);
    K[54] = Ops::fmac(w11, 8.1, Ops::fmac(w3, 8.1, m11));
  }
  template <class Ops> __device__ __forceinline__ static void mass_upper(const typename Ops::T& vol, typename Ops::T* K) {
    const typename Ops::T m0 = Ops::mulc(vol, 0.01130952380952381);
    const typename Ops::T m1 = Ops::mulc(vol, 0.001636904761904762);
    const typename Ops::T m2 = Ops::mulc(vol, 0.0026785714285714286);
    const typename Ops::T m3 = Ops::mulc(vol, 0.0040178571428571425);
    const typename Ops::T m4 = Ops::mulc(vol, 0.005357142857142857);
    const typename Ops::T m5 = Ops::mulc(vol, 0.08035714285714286);
    const typename Ops::T m6 = Ops::mulc(vol, -0.028125);
    const typename Ops::T m7 = Ops::mulc(vol, 0.04017857142857143);
    const typename Ops::T m8 = Ops::mulc(vol, -0.020089285714285716);
    const typename Ops::T m9 = Ops::mulc(vol, -0.008035714285714285);
    const typename Ops::T m10 = Ops::mulc(vol, 0.024107142857142858);
    const typename Ops::T m11 = Ops::mulc(vol, 0.2892857142857143);
    K[0] = m0;
    K[1] = m1;
    K[2] = m1;
    K[3] = m2;
    K[4] = Ops::zero();
    K[5] = m2;
    K[6] = Ops::zero();
    K[7] = m3;
    K[8] = m3;
    K[9] = m4;
    K[10] = m0;
    K[11] = m1;
    K[12] = Ops::zero();
    K[13] = m2;
    K[14] = m3;
    K[15] = m3;
    K[16] = m2;
    K[17] = Ops::zero();
    K[18] = m4;
    K[19] = m0;
    K[20] = m3;
    K[21] = m3;
    K[22] = Ops::zero();
    K[23] = m2;
    K[24] = Ops::zero();
    K[25] = m2;
    K[26] = m4;
    K[27] = m5;
    K[28] = m6;
    K[29] = m7;
    K[30] = m8;
    K[31] = m8;
    K[32] = m9;
    K[33] = m10;
    K[34] = m5;
    K[35] = m8;
    K[36] = m9;
    K[37] = m7;
    K[38] = m8;
    K[39] = m10;
    K[40] = m5;
    K[41] = m6;
    K[42] = m9;
    K[43] = m8;
    K[44] = m10;
    K[45] = m5;
    K[46] = m8;
    K[47] = m7;
    K[48] = m10;
    K[49] = m5;
    K[50] = m6;
    K[51] = m10;
    K[52] = m5;
    K[53] = m10;
    K[54] = m11;
  }
  template <class Ops, bool STIFF, bool MASS> __device__ __forceinline__ static void action_upper(const typename Ops::T* Lam, const typename Ops::T& vol, const typename Ops::T* x, typename Ops::T* y) {
    typename Ops::T k;
    if constexpr (STIFF && MASS) {
      const typename Ops::T w0 = Ops::add(Lam[0], Lam[1]);
      const typename Ops::T w1 = Ops::add(Lam[2], Lam[4]);
      const typename Ops::T w2 = Ops::add(Lam[1], Lam[4]);
      const typename Ops::T w3 = Ops::add(Lam[5], w1);
      const typename Ops::T w4 = Ops::add(Lam[2], w0);
      const typename Ops::T w5 = Ops::add(Lam[3], w2);
      const typename Ops::T w6 = Ops::fmac(w3, 0.5, Lam[1]);
      const typename Ops::T w7 = Ops::fmac(w5, 0.5, Lam[2]);
      const typename Ops::T w8 = Ops::fmac(w4, 0.5, Lam[4]);
      const typename Ops::T w9 = Ops::add(Lam[0], Lam[5]);
      const typename Ops::T w10 = Ops::add(Lam[3], Lam[5]);
      const typename Ops::T w11 = Ops::add(Lam[3], w0);
      const typename Ops::T w12 = Ops::add(Lam[1], Lam[2]);
      const typename Ops::T w13 = Ops::add(Lam[2], w9);
      const typename Ops::T w14 = Ops::add(Lam[4], w10);
      const typename Ops::T m0 = Ops::mulc(vol, 0.01130952380952381);
      const typename Ops::T m1 = Ops::mulc(vol, 0.001636904761904762);
      const typename Ops::T m2 = Ops::mulc(vol, 0.0026785714285714286);
      const typename Ops::T m3 = Ops::mulc(vol, 0.0040178571428571425);
      const typename Ops::T m4 = Ops::mulc(vol, 0.005357142857142857);
      const typename Ops::T m5 = Ops::mulc(vol, 0.08035714285714286);
      const typename Ops::T m6 = Ops::mulc(vol, -0.028125);
      const typename Ops::T m7 = Ops::mulc(vol, 0.04017857142857143);
      const typename Ops::T m8 = Ops::mulc(vol, -0.020089285714285716);
      const typename Ops::T m9 = Ops::mulc(vol, -0.008035714285714285);
      const typename Ops::T m10 = Ops::mulc(vol, 0.024107142857142858);
      const typename Ops::T m11 = Ops::mulc(vol, 0.2892857142857143);
      { k = Ops::fmac(Lam[0], 0.85, m0); y[0] = Ops::mul(k, x[0]); }
      { k = Ops::fmac(Lam[1], 0.175, m1); y[0] = Ops::fma3(k, x[1], y[0]); y[1] = Ops::mul(k, x[0]); }
      { k = Ops::fmac(Lam[2], 0.175, m1); y[0] = Ops::fma3(k, x[2], y[0]); y[2] = Ops::mul(k, x[0]); }
      { k = Ops::fmac(Lam[1], 1.425, Ops::fmac(Lam[0], 0.075, m2)); y[0] = Ops::fma3(k, x[3], y[0]); y[3] = Ops::mul(k, x[0]); }
      { k = Ops::fmac(Lam[1], -0.6, Ops::mulc(Lam[0], 0.075)); y[0] = Ops::fma3(k, x[4], y[0]); y[4] = Ops::mul(k, x[0]); }
      { k = Ops::fmac(Lam[2], 1.425, Ops::fmac(Lam[0], 0.075, m2)); y[0] = Ops::fma3(k, x[5], y[0]); y[5] = Ops::mul(k, x[0]); }
      { k = Ops::fmac(Lam[2], -0.6, Ops::mulc(Lam[0], 0.075)); y[0] = Ops::fma3(k, x[6], y[0]); y[6] = Ops::mul(k, x[0]); }
      { k = Ops::fmac(w12, 0.075, m3); y[0] = Ops::fma3(k, x[7], y[0]); y[7] = Ops::mul(k, x[0]); }
      { k = Ops::fmac(w12, 0.075, m3); y[0] = Ops::fma3(k, x[8], y[0]); y[8] = Ops::mul(k, x[0]); }
      { k = Ops::fmac(w4, 0.225, m4); y[0] = Ops::fma3(k, x[9], y[0]); y[9] = Ops::mul(k, x[0]); }
      { k = Ops::fmac(Lam[3], 0.85, m0); y[1] = Ops::fma3(k, x[1], y[1]); }
      { k = Ops::fmac(Lam[4], 0.175, m1); y[1] = Ops::fma3(k, x[2], y[1]); y[2] = Ops::fma3(k, x[1], y[2]); }
      { k = Ops::fmac(Lam[3], 0.075, Ops::mulc(Lam[1], -0.6)); y[1] = Ops::fma3(k, x[3], y[1]); y[3] = Ops::fma3(k, x[1], y[3]); }
      { k = Ops::fmac(Lam[3], 0.075, Ops::fmac(Lam[1], 1.425, m2)); y[1] = Ops::fma3(k, x[4], y[1]); y[4] = Ops::fma3(k, x[1], y[4]); }
      { k = Ops::fmac(w2, 0.075, m3); y[1] = Ops::fma3(k, x[5], y[1]); y[5] = Ops::fma3(k, x[1], y[5]); }
      { k = Ops::fmac(w2, 0.075, m3); y[1] = Ops::fma3(k, x[6], y[1]); y[6] = Ops::fma3(k, x[1], y[6]); }
      { k = Ops::fmac(Lam[4], 1.425, Ops::fmac(Lam[3], 0.075, m2)); y[1] = Ops::fma3(k, x[7], y[1]); y[7] = Ops::fma3(k, x[1], y[7]); }
      { k = Ops::fmac(Lam[4], -0.6, Ops::mulc(Lam[3], 0.075)); y[1] = Ops::fma3(k, x[8], y[1]); y[8] = Ops::fma3(k, x[1], y[8]); }
      { k = Ops::fmac(w5, 0.225, m4); y[1] = Ops::fma3(k, x[9], y[1]); y[9] = Ops::fma3(k, x[1], y[9]); }
      { k = Ops::fmac(Lam[5], 0.85, m0); y[2] = Ops::fma3(k, x[2], y[2]); }
      { k = Ops::fmac(w1, 0.075, m3); y[2] = Ops::fma3(k, x[3], y[2]); y[3] = Ops::fma3(k, x[2], y[3]); }
      { k = Ops::fmac(w1, 0.075, m3); y[2] = Ops::fma3(k, x[4], y[2]); y[4] = Ops::fma3(k, x[2], y[4]); }
      { k = Ops::fmac(Lam[5], 0.075, Ops::mulc(Lam[2], -0.6)); y[2] = Ops::fma3(k, x[5], y[2]); y[5] = Ops::fma3(k, x[2], y[5]); }
      { k = Ops::fmac(Lam[5], 0.075, Ops::fmac(Lam[2], 1.425, m2)); y[2] = Ops::fma3(k, x[6], y[2]); y[6] = Ops::fma3(k, x[2], y[6]); }
      { k = Ops::fmac(Lam[5], 0.075, Ops::mulc(Lam[4], -0.6)); y[2] = Ops::fma3(k, x[7], y[2]); y[7] = Ops::fma3(k, x[2], y[7]); }
      { k = Ops::fmac(Lam[5], 0.075, Ops::fmac(Lam[4], 1.425, m2)); y[2] = Ops::fma3(k, x[8], y[2]); y[8] = Ops::fma3(k, x[2], y[8]); }
      { k = Ops::fmac(w3, 0.225, m4); y[2] = Ops::fma3(k, x[9], y[2]); y[9] = Ops::fma3(k, x[2], y[9]); }
      { k = Ops::fmac(w11, 3.375, m5); y[3] = Ops::fma3(k, x[3], y[3]); }
      { k = Ops::fmac(Lam[3], -0.675, Ops::fmac(Lam[1], 1.35, Ops::fmac(Lam[0], -0.675, m6))); y[3] = Ops::fma3(k, x[4], y[3]); y[4] = Ops::fma3(k, x[3], y[4]); }
      { k = Ops::fmac(w8, 3.375, m7); y[3] = Ops::fma3(k, x[5], y[3]); y[5] = Ops::fma3(k, x[3], y[5]); }
      { k = Ops::fmac(w8, -0.675, m8); y[3] = Ops::fma3(k, x[6], y[3]); y[6] = Ops::fma3(k, x[3], y[6]); }
      { k = Ops::fmac(w7, -0.675, m8); y[3] = Ops::fma3(k, x[7], y[3]); y[7] = Ops::fma3(k, x[3], y[7]); }
      { k = Ops::fmac(w7, -0.675, m9); y[3] = Ops::fma3(k, x[8], y[3]); y[8] = Ops::fma3(k, x[3], y[8]); }
      { k = Ops::fmac(w7, 4.05, m10); y[3] = Ops::fma3(k, x[9], y[3]); y[9] = Ops::fma3(k, x[3], y[9]); }
      { k = Ops::fmac(w11, 3.375, m5); y[4] = Ops::fma3(k, x[4], y[4]); }
      { k = Ops::fmac(w8, -0.675, m8); y[4] = Ops::fma3(k, x[5], y[4]); y[5] = Ops::fma3(k, x[4], y[5]); }
      { k = Ops::fmac(w8, -0.675, m9); y[4] = Ops::fma3(k, x[6], y[4]); y[6] = Ops::fma3(k, x[4], y[6]); }
      { k = Ops::fmac(w7, 3.375, m7); y[4] = Ops::fma3(k, x[7], y[4]); y[7] = Ops::fma3(k, x[4], y[7]); }
      { k = Ops::fmac(w7, -0.675, m8); y[4] = Ops::fma3(k, x[8], y[4]); y[8] = Ops::fma3(k, x[4], y[8]); }
      { k = Ops::fmac(w8, 4.05, m10); y[4] = Ops::fma3(k, x[9], y[4]); y[9] = Ops::fma3(k, x[4], y[9]); }
      { k = Ops::fmac(w13, 3.375, m5); y[5] = Ops::fma3(k, x[5], y[5]); }
      { k = Ops::fmac(w9, -0.675, Ops::fmac(Lam[2], 1.35, m6)); y[5] = Ops::fma3(k, x[6], y[5]); y[6] = Ops::fma3(k, x[5], y[6]); }
      { k = Ops::fmac(w6, -0.675, m9); y[5] = Ops::fma3(k, x[7], y[5]); y[7] = Ops::fma3(k, x[5], y[7]); }
      { k = Ops::fmac(w6, -0.675, m8); y[5] = Ops::fma3(k, x[8], y[5]); y[8] = Ops::fma3(k, x[5], y[8]); }
      { k = Ops::fmac(w6, 4.05, m10); y[5] = Ops::fma3(k, x[9], y[5]); y[9] = Ops::fma3(k, x[5], y[9]); }
      { k = Ops::fmac(w13, 3.375, m5); y[6] = Ops::fma3(k, x[6], y[6]); }
      { k = Ops::fmac(w6, -0.675, m8); y[6] = Ops::fma3(k, x[7], y[6]); y[7] = Ops::fma3(k, x[6], y[7]); }
      { k = Ops::fmac(w6, 3.375, m7); y[6] = Ops::fma3(k, x[8], y[6]); y[8] = Ops::fma3(k, x[6], y[8]); }
      { k = Ops::fmac(w8, 4.05, m10); y[6] = Ops::fma3(k, x[9], y[6]); y[9] = Ops::fma3(k, x[6], y[9]); }
      { k = Ops::fmac(w14, 3.375, m5); y[7] = Ops::fma3(k, x[7], y[7]); }
      { k = Ops::fmac(w10, -0.675, Ops::fmac(Lam[4], 1.35, m6)); y[7] = Ops::fma3(k, x[8], y[7]); y[8] = Ops::fma3(k, x[7], y[8]); }
      { k = Ops::fmac(w6, 4.05, m10); y[7] = Ops::fma3(k, x[9], y[7]); y[9] = Ops::fma3(k, x[7], y[9]); }
      { k = Ops::fmac(w14, 3.375, m5); y[8] = Ops::fma3(k, x[8], y[8]); }
      { k = Ops::fmac(w7, 4.05, m10); y[8] = Ops::fma3(k, x[9], y[8]); y[9] = Ops::fma3(k, x[8], y[9]); }
      { k = Ops::fmac(w11, 8.1, Ops::fmac(w3, 8.1, m11)); y[9] = Ops::fma3(k, x[9], y[9]); }
    }
    else if constexpr (STIFF) {
      const typename Ops::T w0 = Ops::add(Lam[0], Lam[1]);
      const typename Ops::T w1 = Ops::add(Lam[2], Lam[4]);
      const typename Ops::T w2 = Ops::add(Lam[1], Lam[4]);
      const typename Ops::T w3 = Ops::add(Lam[5], w1);
      const typename Ops::T w4 = Ops::add(Lam[2], w0);
      const typename Ops::T w5 = Ops::add(Lam[3], w2);
      const typename Ops::T w6 = Ops::fmac(w3, 0.5, Lam[1]);
      const typename Ops::T w7 = Ops::fmac(w5, 0.5, Lam[2]);
      const typename Ops::T w8 = Ops::fmac(w4, 0.5, Lam[4]);
      const typename Ops::T w9 = Ops::add(Lam[0], Lam[5]);
      const typename Ops::T w10 = Ops::add(Lam[3], Lam[5]);
      const typename Ops::T w11 = Ops::add(Lam[3], w0);
      const typename Ops::T w12 = Ops::add(Lam[1], Lam[2]);
      const typename Ops::T w13 = Ops::add(Lam[2], w9);
      const typename Ops::T w14 = Ops::add(Lam[4], w10);
      { k = Ops::mulc(Lam[0], 0.85); y[0] = Ops::mul(k, x[0]); }
      { k = Ops::mulc(Lam[1], 0.175); y[0] = Ops::fma3(k, x[1], y[0]); y[1] = Ops::mul(k, x[0]); }
      { k = Ops::mulc(Lam[2], 0.175); y[0] = Ops::fma3(k, x[2], y[0]); y[2] = Ops::mul(k, x[0]); }
      { k = Ops::fmac(Lam[1], 1.425, Ops::mulc(Lam[0], 0.075)); y[0] = Ops::fma3(k, x[3], y[0]); y[3] = Ops::mul(k, x[0]); }
      { k = Ops::fmac(Lam[1], -0.6, Ops::mulc(Lam[0], 0.075)); y[0] = Ops::fma3(k, x[4], y[0]); y[4] = Ops::mul(k, x[0]); }
      { k = Ops::fmac(Lam[2], 1.425, Ops::mulc(Lam[0], 0.075)); y[0] = Ops::fma3(k, x[5], y[0]); y[5] = Ops::mul(k, x[0]); }
      { k = Ops::fmac(Lam[2], -0.6, Ops::mulc(Lam[0], 0.075)); y[0] = Ops::fma3(k, x[6], y[0]); y[6] = Ops::mul(k, x[0]); }
      { k = Ops::mulc(w12, 0.075); y[0] = Ops::fma3(k, x[7], y[0]); y[7] = Ops::mul(k, x[0]); }
      { k = Ops::mulc(w12, 0.075); y[0] = Ops::fma3(k, x[8], y[0]); y[8] = Ops::mul(k, x[0]); }
      { k = Ops::mulc(w4, 0.225); y[0] = Ops::fma3(k, x[9], y[0]); y[9] = Ops::mul(k, x[0]); }
      { k = Ops::mulc(Lam[3], 0.85); y[1] = Ops::fma3(k, x[1], y[1]); }
      { k = Ops::mulc(Lam[4], 0.175); y[1] = Ops::fma3(k, x[2], y[1]); y[2] = Ops::fma3(k, x[1], y[2]); }
      { k = Ops::fmac(Lam[3], 0.075, Ops::mulc(Lam[1], -0.6)); y[1] = Ops::fma3(k, x[3], y[1]); y[3] = Ops::fma3(k, x[1], y[3]); }
      { k = Ops::fmac(Lam[3], 0.075, Ops::mulc(Lam[1], 1.425)); y[1] = Ops::fma3(k, x[4], y[1]); y[4] = Ops::fma3(k, x[1], y[4]); }
      { k = Ops::mulc(w2, 0.075); y[1] = Ops::fma3(k, x[5], y[1]); y[5] = Ops::fma3(k, x[1], y[5]); }
      { k = Ops::mulc(w2, 0.075); y[1] = Ops::fma3(k, x[6], y[1]); y[6] = Ops::fma3(k, x[1], y[6]); }
      { k = Ops::fmac(Lam[4], 1.425, Ops::mulc(Lam[3], 0.075)); y[1] = Ops::fma3(k, x[7], y[1]); y[7] = Ops::fma3(k, x[1], y[7]); }
      { k = Ops::fmac(Lam[4], -0.6, Ops::mulc(Lam[3], 0.075)); y[1] = Ops::fma3(k, x[8], y[1]); y[8] = Ops::fma3(k, x[1], y[8]); }
      { k = Ops::mulc(w5, 0.225); y[1] = Ops::fma3(k, x[9], y[1]); y[9] = Ops::fma3(k, x[1], y[9]); }
      { k = Ops::mulc(Lam[5], 0.85); y[2] = Ops::fma3(k, x[2], y[2]); }
      { k = Ops::mulc(w1, 0.075); y[2] = Ops::fma3(k, x[3], y[2]); y[3] = Ops::fma3(k, x[2], y[3]); }
      { k = Ops::mulc(w1, 0.075); y[2] = Ops::fma3(k, x[4], y[2]); y[4] = Ops::fma3(k, x[2], y[4]); }
      { k = Ops::fmac(Lam[5], 0.075, Ops::mulc(Lam[2], -0.6)); y[2] = Ops::fma3(k, x[5], y[2]); y[5] = Ops::fma3(k, x[2], y[5]); }
      { k = Ops::fmac(Lam[5], 0.075, Ops::mulc(Lam[2], 1.425)); y[2] = Ops::fma3(k, x[6], y[2]); y[6] = Ops::fma3(k, x[2], y[6]); }
      { k = Ops::fmac(Lam[5], 0.075, Ops::mulc(Lam[4], -0.6)); y[2] = Ops::fma3(k, x[7], y[2]); y[7] = Ops::fma3(k, x[2], y[7]); }
      { k = Ops::fmac(Lam[5], 0.075, Ops::mulc(Lam[4], 1.425)); y[2] = Ops::fma3(k, x[8], y[2]); y[8] = Ops::fma3(k, x[2], y[8]); }
      { k = Ops::mulc(w3, 0.225); y[2] = Ops::fma3(k, x[9], y[2]); y[9] = Ops::fma3(k, x[2], y[9]); }
      { k = Ops::mulc(w11, 3.375); y[3] = Ops::fma3(k, x[3], y[3]); }
      { k = Ops::fmac(Lam[3], -0.675, Ops::fmac(Lam[1], 1.35, Ops::mulc(Lam[0], -0.675))); y[3] = Ops::fma3(k, x[4], y[3]); y[4] = Ops::fma3(k, x[3], y[4]); }
      { k = Ops::mulc(w8, 3.375); y[3] = Ops::fma3(k, x[5], y[3]); y[5] = Ops::fma3(k, x[3], y[5]); }
      { k = Ops::mulc(w8, -0.675); y[3] = Ops::fma3(k, x[6], y[3]); y[6] = Ops::fma3(k, x[3], y[6]); }
      { k = Ops::mulc(w7, -0.675); y[3] = Ops::fma3(k, x[7], y[3]); y[7] = Ops::fma3(k, x[3], y[7]); }
      { k = Ops::mulc(w7, -0.675); y[3] = Ops::fma3(k, x[8], y[3]); y[8] = Ops::fma3(k, x[3], y[8]); }
      { k = Ops::mulc(w7, 4.05); y[3] = Ops::fma3(k, x[9], y[3]); y[9] = Ops::fma3(k, x[3], y[9]); }
      { k = Ops::mulc(w11, 3.375); y[4] = Ops::fma3(k, x[4], y[4]); }
      { k = Ops::mulc(w8, -0.675); y[4] = Ops::fma3(k, x[5], y[4]); y[5] = Ops::fma3(k, x[4], y[5]); }
      { k = Ops::mulc(w8, -0.675); y[4] = Ops::fma3(k, x[6], y[4]); y[6] = Ops::fma3(k, x[4], y[6]); }
      { k = Ops::mulc(w7, 3.375); y[4] = Ops::fma3(k, x[7], y[4]); y[7] = Ops::fma3(k, x[4], y[7]); }
      { k = Ops::mulc(w7, -0.675); y[4] = Ops::fma3(k, x[8], y[4]); y[8] = Ops::fma3(k, x[4], y[8]); }
      { k = Ops::mulc(w8, 4.05); y[4] = Ops::fma3(k, x[9], y[4]); y[9] = Ops::fma3(k, x[4], y[9]); }
      { k = Ops::mulc(w13, 3.375); y[5] = Ops::fma3(k, x[5], y[5]); }
      { k = Ops::fmac(w9, -0.675, Ops::mulc(Lam[2], 1.35)); y[5] = Ops::fma3(k, x[6], y[5]); y[6] = Ops::fma3(k, x[5], y[6]); }
      { k = Ops::mulc(w6, -0.675); y[5] = Ops::fma3(k, x[7], y[5]); y[7] = Ops::fma3(k, x[5], y[7]); }
      { k = Ops::mulc(w6, -0.675); y[5] = Ops::fma3(k, x[8], y[5]); y[8] = Ops::fma3(k, x[5], y[8]); }
      { k = Ops::mulc(w6, 4.05); y[5] = Ops::fma3(k, x[9], y[5]); y[9] = Ops::fma3(k, x[5], y[9]); }
      { k = Ops::mulc(w13, 3.375); y[6] = Ops::fma3(k, x[6], y[6]); }
      { k = Ops::mulc(w6, -0.675); y[6] = Ops::fma3(k, x[7], y[6]); y[7] = Ops::fma3(k, x[6], y[7]); }
      { k = Ops::mulc(w6, 3.375); y[6] = Ops::fma3(k, x[8], y[6]); y[8] = Ops::fma3(k, x[6], y[8]); }
      { k = Ops::mulc(w8, 4.05); y[6] = Ops::fma3(k, x[9], y[6]); y[9] = Ops::fma3(k, x[6], y[9]); }
      { k = Ops::mulc(w14, 3.375); y[7] = Ops::fma3(k, x[7], y[7]); }
      { k = Ops::fmac(w10, -0.675, Ops::mulc(Lam[4], 1.35)); y[7] = Ops::fma3(k, x[8], y[7]); y[8] = Ops::fma3(k, x[7], y[8]); }
      { k = Ops::mulc(w6, 4.05); y[7] = Ops::fma3(k, x[9], y[7]); y[9] = Ops::fma3(k, x[7], y[9]); }
      { k = Ops::mulc(w14, 3.375); y[8] = Ops::fma3(k, x[8], y[8]); }
      { k = Ops::mulc(w7, 4.05); y[8] = Ops::fma3(k, x[9], y[8]); y[9] = Ops::fma3(k, x[8], y[9]); }
      { k = Ops::fmac(w11, 8.1, Ops::mulc(w3, 8.1)); y[9] = Ops::fma3(k, x[9], y[9]); }
    }
    else if constexpr (MASS) {
      const typename Ops::T m0 = Ops::mulc(vol, 0.01130952380952381);
      const typename Ops::T m1 = Ops::mulc(vol, 0.001636904761904762);
      const typename Ops::T m2 = Ops::mulc(vol, 0.0026785714285714286);
      const typename Ops::T m3 = Ops::mulc(vol, 0.0040178571428571425);
      const typename Ops::T m4 = Ops::mulc(vol, 0.005357142857142857);
      const typename Ops::T m5 = Ops::mulc(vol, 0.08035714285714286);
      const typename Ops::T m6 = Ops::mulc(vol, -0.028125);
      const typename Ops::T m7 = Ops::mulc(vol, 0.04017857142857143);
      const typename Ops::T m8 = Ops::mulc(vol, -0.020089285714285716);
      const typename Ops::T m9 = Ops::mulc(vol, -0.008035714285714285);
      const typename Ops::T m10 = Ops::mulc(vol, 0.024107142857142858);
      const typename Ops::T m11 = Ops::mulc(vol, 0.2892857142857143);
      { k = m0; y[0] = Ops::mul(k, x[0]); }
      { k = m1; y[0] = Ops::fma3(k, x[1], y[0]); y[1] = Ops::mul(k, x[0]); }
      { k = m1; y[0] = Ops::fma3(k, x[2], y[0]); y[2] = Ops::mul(k, x[0]); }
      { k = m2; y[0] = Ops::fma3(k, x[3], y[0]); y[3] = Ops::mul(k, x[0]); }
      { k = m2; y[0] = Ops::fma3(k, x[5], y[0]); y[5] = Ops::mul(k, x[0]); }
      { k = m3; y[0] = Ops::fma3(k, x[7], y[0]); y[7] = Ops::mul(k, x[0]); }
      { k = m3; y[0] = Ops::fma3(k, x[8], y[0]); y[8] = Ops::mul(k, x[0]); }
      { k = m4; y[0] = Ops::fma3(k, x[9], y[0]); y[9] = Ops::mul(k, x[0]); }
      { k = m0; y[1] = Ops::fma3(k, x[1], y[1]); }
      { k = m1; y[1] = Ops::fma3(k, x[2], y[1]); y[2] = Ops::fma3(k, x[1], y[2]); }
      { k = m2; y[1] = Ops::fma3(k, x[4], y[1]); y[4] = Ops::mul(k, x[1]); }
      { k = m3; y[1] = Ops::fma3(k, x[5], y[1]); y[5] = Ops::fma3(k, x[1], y[5]); }
      { k = m3; y[1] = Ops::fma3(k, x[6], y[1]); y[6] = Ops::mul(k, x[1]); }
      { k = m2; y[1] = Ops::fma3(k, x[7], y[1]); y[7] = Ops::fma3(k, x[1], y[7]); }
      { k = m4; y[1] = Ops::fma3(k, x[9], y[1]); y[9] = Ops::fma3(k, x[1], y[9]); }
      { k = m0; y[2] = Ops::fma3(k, x[2], y[2]); }
      { k = m3; y[2] = Ops::fma3(k, x[3], y[2]); y[3] = Ops::fma3(k, x[2], y[3]); }
      { k = m3; y[2] = Ops::fma3(k, x[4], y[2]); y[4] = Ops::fma3(k, x[2], y[4]); }
      { k = m2; y[2] = Ops::fma3(k, x[6], y[2]); y[6] = Ops::fma3(k, x[2], y[6]); }
      { k = m2; y[2] = Ops::fma3(k, x[8], y[2]); y[8] = Ops::fma3(k, x[2], y[8]); }
      { k = m4; y[2] = Ops::fma3(k, x[9], y[2]); y[9] = Ops::fma3(k, x[2], y[9]); }
      { k = m5; y[3] = Ops::fma3(k, x[3], y[3]); }
      { k = m6; y[3] = Ops::fma3(k, x[4], y[3]); y[4] = Ops::fma3(k, x[3], y[4]); }
      { k = m7; y[3] = Ops::fma3(k, x[5], y[3]); y[5] = Ops::fma3(k, x[3], y[5]); }
      { k = m8; y[3] = Ops::fma3(k, x[6], y[3]); y[6] = Ops::fma3(k, x[3], y[6]); }
      { k = m8; y[3] = Ops::fma3(k, x[7], y[3]); y[7] = Ops::fma3(k, x[3], y[7]); }
      { k = m9; y[3] = Ops::fma3(k, x[8], y[3]); y[8] = Ops::fma3(k, x[3], y[8]); }
      { k = m10; y[3] = Ops::fma3(k, x[9], y[3]); y[9] = Ops::fma3(k, x[3], y[9]); }
      { k = m5; y[4] = Ops::fma3(k, x[4], y[4]); }
      { k = m8; y[4] = Ops::fma3(k, x[5], y[4]); y[5] = Ops::fma3(k, x[4], y[5]); }
      { k = m9; y[4] = Ops::fma3(k, x[6], y[4]); y[6] = Ops::fma3(k, x[4], y[6]); }
      { k = m7; y[4] = Ops::fma3(k, x[7], y[4]); y[7] = Ops::fma3(k, x[4], y[7]); }
      { k = m8; y[4] = Ops::fma3(k, x[8], y[4]); y[8] = Ops::fma3(k, x[4], y[8]); }
      { k = m10; y[4] = Ops::fma3(k, x[9], y[4]); y[9] = Ops::fma3(k, x[4], y[9]); }
      { k = m5; y[5] = Ops::fma3(k, x[5], y[5]); }
      { k = m6; y[5] = Ops::fma3(k, x[6], y[5]); y[6] = Ops::fma3(k, x[5], y[6]); }
      { k = m9; y[5] = Ops::fma3(k, x[7], y[5]); y[7] = Ops::fma3(k, x[5], y[7]); }
      { k = m8; y[5] = Ops::fma3(k, x[8], y[5]); y[8] = Ops::fma3(k, x[5], y[8]); }
      { k = m10; y[5] = Ops::fma3(k, x[9], y[5]); y[9] = Ops::fma3(k, x[5], y[9]); }
      { k = m5; y[6] = Ops::fma3(k, x[6], y[6]); }
      { k = m8; y[6] = Ops::fma3(k, x[7], y[6]); y[7] = Ops::fma3(k, x[6], y[7]); }
      { k = m7; y[6] = Ops::fma3(k, x[8], y[6]); y[8] = Ops::fma3(k, x[6], y[8]); }
      { k = m10; y[6] = Ops::fma3(k, x[9], y[6]); y[9] = Ops::fma3(k, x[6], y[9]); }
      { k = m5; y[7] = Ops::fma3(k, x[7], y[7]); }
      { k = m6; y[7] = Ops::fma3(k, x[8], y[7]); y[8] = Ops::fma3(k, x[7], y[8]); }
      { k = m10; y[7] = Ops::fma3(k, x[9], y[7]); y[9] = Ops::fma3(k, x[7], y[9]); }
      { k = m5; y[8] = Ops::fma3(k, x[8], y[8]); }
      { k = m10; y[8] = Ops::fma3(k, x[9], y[8]); y[9] = Ops::fma3(k, x[8], y[9]); }
      { k = m11; y[9] = Ops::fma3(k, x[9], y[9]); }
    }
  }
  __host__ __device__ static constexpr int upper_index(int i, int j) {
    return i <= j ? i * 10 - (i * (i - 1)) / 2 + (j - i) : j * 10 - (j * (j - 1)) / 2 + (i - j);
  }
};

// ---- P4 Lagrange on the triangle (15 nodes) ----
template <> struct Elem<2, 4> {
  static constexpr int ND = 15;
  static constexpr int NUP = 120;
  static constexpr int NLAM = 6;
  static constexpr int STIFF_TERMS = 414;
  // K[u] for u over the upper triangle (i <= j), row-major; Lam[k] over pairs (m <= n)
  static constexpr int STIFF_OPS = 290;  // after rewriting
  template <class Ops> __device__ __forceinline__ static void stiffness_upper(const typename Ops::T* Lam, typename Ops::T* K) {
    const typename Ops::T w0 = Ops::add(Lam[1], Lam[2]);
    const typename Ops::T w1 = Ops::add(Lam[1], Lam[4]);
    const typename Ops::T w2 = Ops::add(Lam[2], Lam[4]);
    const typename Ops::T w3 = Ops::add(Lam[0], w0);
    const typename Ops::T w4 = Ops::add(Lam[3], Lam[4]);
    const typename Ops::T w5 = Ops::add(Lam[3], w1);
    const typename Ops::T w6 = Ops::add(Lam[5], w2);
    const typename Ops::T w7 = Ops::add(Lam[0], Lam[1]);
    const typename Ops::T w8 = Ops::add(Lam[0], Lam[2]);
    const typename Ops::T w9 = Ops::add(Lam[0], Lam[3]);
    const typename Ops::T w10 = Ops::add(Lam[0], Lam[5]);
    const typename Ops::T w11 = Ops::add(Lam[1], Lam[3]);
    const typename Ops::T w12 = Ops::add(Lam[2], Lam[5]);
    const typename Ops::T w13 = Ops::add(Lam[3], Lam[5]);
    const typename Ops::T w14 = Ops::add(Lam[4], Lam[5]);
    const typename Ops::T w15 = Ops::add(Lam[5], w3);
    const typename Ops::T w16 = Ops::add(w4, w15);
    const typename Ops::T w17 = Ops::fmac(Lam[4], 2.0930232558139537, Lam[0]);
    const typename Ops::T w18 = Ops::fmac(Lam[4], 1.7692307692307692, Lam[0]);
    const typename Ops::T w19 = Ops::fmac(w0, 0.2, Lam[0]);
    const typename Ops::T w20 = Ops::fmac(Lam[5], 0.4777777777777778, Lam[1]);
    const typename Ops::T w21 = Ops::fmac(Lam[5], 0.5652173913043478, Lam[1]);
    const typename Ops::T w22 = Ops::fmac(w2, 0.5, Lam[1]);
    const typename Ops::T w23 = Ops::fmac(w6, 0.631578947368421, Lam[1]);
    const typename Ops::T w24 = Ops::fmac(w6, 0.4, Lam[1]);
    const typename Ops::T w25 = Ops::fmac(Lam[3], 0.4777777777777778, Lam[2]);
    const typename Ops::T w26 = Ops::fmac(Lam[3], 0.5652173913043478, Lam[2]);
    const typename Ops::T w27 = Ops::fmac(w1, 0.5, Lam[2]);
    const typename Ops::T w28 = Ops::fmac(w5, 0.631578947368421, Lam[2]);
    const typename Ops::T w29 = Ops::fmac(w5, 0.4, Lam[2]);
    const typename Ops::T w30 = Ops::fmac(w1, 0.2, Lam[3]);
    const typename Ops::T w31 = Ops::fmac(w0, 0.5, Lam[4]);
    const typename Ops::T w32 = Ops::fmac(w3, 0.631578947368421, Lam[4]);
    const typename Ops::T w33 = Ops::fmac(w3, 0.4, Lam[4]);
    const typename Ops::T w34 = Ops::fmac(w2, 0.2, Lam[5]);
    const typename Ops::T w35 = Ops::fmac(w18, 1.4444444444444444, w0);
    const typename Ops::T w36 = Ops::fmac(w26, 2.5555555555555554, w1);
    const typename Ops::T w37 = Ops::fmac(w21, 2.5555555555555554, w2);
    K[0] = Ops::mulc(Lam[0], 0.746031746031746);
    K[1] = Ops::mulc(Lam[1], -0.11322751322751323);
    K[2] = Ops::mulc(Lam[2], -0.11322751322751323);
    K[3] = Ops::fmac(Lam[1], 1.5576719576719578, Ops::mulc(Lam[0], 0.25396825396825395));
    K[4] = Ops::fmac(Lam[1], -0.8507936507936508, Ops::mulc(Lam[0], 0.08465608465608465));
    K[5] = Ops::fmac(Lam[1], 0.40634920634920635, Ops::mulc(Lam[0], -0.08465608465608465));
    K[6] = Ops::fmac(Lam[2], 1.5576719576719578, Ops::mulc(Lam[0], 0.25396825396825395));
    K[7] = Ops::fmac(Lam[2], -0.8507936507936508, Ops::mulc(Lam[0], 0.08465608465608465));
    K[8] = Ops::fmac(Lam[2], 0.40634920634920635, Ops::mulc(Lam[0], -0.08465608465608465));
    K[9] = Ops::mulc(w0, -0.08465608465608465);
    K[10] = Ops::mulc(w0, -0.08465608465608465);
    K[11] = Ops::mulc(w0, -0.08465608465608465);
    K[12] = Ops::fmac(w0, 0.6349206349206349, Ops::mulc(Lam[0], 0.4656084656084656));
    K[13] = Ops::mulc(w19, -0.21164021164021163);
    K[14] = Ops::mulc(w19, -0.21164021164021163);
    K[15] = Ops::mulc(Lam[3], 0.746031746031746);
    K[16] = Ops::mulc(Lam[4], -0.11322751322751323);
    K[17] = Ops::fmac(Lam[3], -0.08465608465608465, Ops::mulc(Lam[1], 0.40634920634920635));
    K[18] = Ops::fmac(Lam[3], 0.08465608465608465, Ops::mulc(Lam[1], -0.8507936507936508));
    K[19] = Ops::fmac(Lam[3], 0.25396825396825395, Ops::mulc(Lam[1], 1.5576719576719578));
    K[20] = Ops::mulc(w1, -0.08465608465608465);
    K[21] = Ops::mulc(w1, -0.08465608465608465);
    K[22] = Ops::mulc(w1, -0.08465608465608465);
    K[23] = Ops::fmac(Lam[4], 1.5576719576719578, Ops::mulc(Lam[3], 0.25396825396825395));
    K[24] = Ops::fmac(Lam[4], -0.8507936507936508, Ops::mulc(Lam[3], 0.08465608465608465));
    K[25] = Ops::fmac(Lam[4], 0.40634920634920635, Ops::mulc(Lam[3], -0.08465608465608465));
    K[26] = Ops::mulc(w30, -0.21164021164021163);
    K[27] = Ops::fmac(w1, 0.6349206349206349, Ops::mulc(Lam[3], 0.4656084656084656));
    K[28] = Ops::mulc(w30, -0.21164021164021163);
    K[29] = Ops::mulc(Lam[5], 0.746031746031746);
    K[30] = Ops::mulc(w2, -0.08465608465608465);
    K[31] = Ops::mulc(w2, -0.08465608465608465);
    K[32] = Ops::mulc(w2, -0.08465608465608465);
    K[33] = Ops::fmac(Lam[5], -0.08465608465608465, Ops::mulc(Lam[2], 0.40634920634920635));
    K[34] = Ops::fmac(Lam[5], 0.08465608465608465, Ops::mulc(Lam[2], -0.8507936507936508));
    K[35] = Ops::fmac(Lam[5], 0.25396825396825395, Ops::mulc(Lam[2], 1.5576719576719578));
    K[36] = Ops::fmac(Lam[5], -0.08465608465608465, Ops::mulc(Lam[4], 0.40634920634920635));
    K[37] = Ops::fmac(Lam[5], 0.08465608465608465, Ops::mulc(Lam[4], -0.8507936507936508));
    K[38] = Ops::fmac(Lam[5], 0.25396825396825395, Ops::mulc(Lam[4], 1.5576719576719578));
    K[39] = Ops::mulc(w34, -0.21164021164021163);
    K[40] = Ops::mulc(w34, -0.21164021164021163);
    K[41] = Ops::fmac(w2, 0.6349206349206349, Ops::mulc(Lam[5], 0.4656084656084656));
    K[42] = Ops::fmac(w11, 4.1989417989417985, Ops::mulc(Lam[0], 3.657142857142857));
    K[43] = Ops::fmac(Lam[3], -1.5238095238095237, Ops::fmac(Lam[1], 1.0497354497354496, Ops::mulc(Lam[0], -1.3206349206349206)));
    K[44] = Ops::fmac(w9, 0.6772486772486772, Ops::mulc(Lam[1], -0.6772486772486772));
    K[45] = Ops::fmac(w31, 4.1989417989417985, Ops::mulc(Lam[0], 1.8285714285714285));
    K[46] = Ops::fmac(w17, -0.728042328042328, Ops::fmac(Lam[2], -0.9312169312169312, Ops::mulc(Lam[1], -0.5925925925925926)));
    K[47] = Ops::fmac(w7, 0.20317460317460317, Ops::fmac(Lam[4], 0.6772486772486772, Ops::mulc(Lam[2], 0.4740740740740741)));
    K[48] = Ops::fmac(w4, 0.20317460317460317, Ops::fmac(Lam[2], 0.6772486772486772, Ops::mulc(Lam[1], 0.4740740740740741)));
    K[49] = Ops::fmac(w4, 0.08465608465608465, Ops::fmac(Lam[2], 0.3047619047619048, Ops::mulc(Lam[1], 0.2201058201058201)));
    K[50] = Ops::fmac(w5, 0.20317460317460317, Ops::mulc(Lam[2], 0.40634920634920635));
    K[51] = Ops::fmac(w28, 5.147089947089947, Ops::mulc(Lam[0], 0.2708994708994709));
    K[52] = Ops::fmac(w4, -0.5417989417989418, Ops::fmac(Lam[2], -0.8126984126984127, Ops::mulc(Lam[0], 0.8126984126984127)));
    K[53] = Ops::fmac(w29, -1.3544973544973544, Ops::mulc(Lam[0], 0.2708994708994709));
    K[54] = Ops::fmac(w9, 4.901587301587302, Ops::mulc(Lam[1], 3.8857142857142857));
    K[55] = Ops::fmac(Lam[3], -1.3206349206349206, Ops::fmac(Lam[1], 1.0497354497354496, Ops::mulc(Lam[0], -1.5238095238095237)));
    K[56] = Ops::fmac(w17, -0.728042328042328, Ops::fmac(Lam[2], -0.5925925925925926, Ops::mulc(Lam[1], -0.9312169312169312)));
    K[57] = Ops::fmac(w31, -0.7873015873015873, Ops::mulc(Lam[0], -0.2920634920634921));
    K[58] = Ops::fmac(w7, 0.08465608465608465, Ops::fmac(Lam[4], 0.3047619047619048, Ops::mulc(Lam[2], 0.2201058201058201)));
    K[59] = Ops::fmac(w25, -1.5238095238095237, Ops::fmac(Lam[4], -0.5925925925925926, Ops::mulc(Lam[1], -0.9312169312169312)));
    K[60] = Ops::fmac(w27, -0.7873015873015873, Ops::mulc(Lam[3], -0.2920634920634921));
    K[61] = Ops::fmac(w11, 0.08465608465608465, Ops::fmac(Lam[4], 0.2201058201058201, Ops::mulc(Lam[2], 0.3047619047619048)));
    K[62] = Ops::fmac(w35, 1.8285714285714285, Ops::mulc(Lam[3], -1.0158730158730158));
    K[63] = Ops::fmac(w36, 1.8285714285714285, Ops::mulc(Lam[0], -1.0158730158730158));
    K[64] = Ops::fmac(w9, -0.6095238095238096, Ops::fmac(w2, -1.4222222222222223, Ops::mulc(Lam[1], -1.0158730158730158)));
    K[65] = Ops::fmac(w7, 4.1989417989417985, Ops::mulc(Lam[3], 3.657142857142857));
    K[66] = Ops::fmac(w8, 0.20317460317460317, Ops::fmac(Lam[4], 0.6772486772486772, Ops::mulc(Lam[1], 0.4740740740740741)));
    K[67] = Ops::fmac(w8, 0.08465608465608465, Ops::fmac(Lam[4], 0.3047619047619048, Ops::mulc(Lam[1], 0.2201058201058201)));
    K[68] = Ops::fmac(w3, 0.20317460317460317, Ops::mulc(Lam[4], 0.40634920634920635));
    K[69] = Ops::fmac(w27, 4.1989417989417985, Ops::mulc(Lam[3], 1.8285714285714285));
    K[70] = Ops::fmac(w25, -1.5238095238095237, Ops::fmac(Lam[4], -0.9312169312169312, Ops::mulc(Lam[1], -0.5925925925925926)));
    K[71] = Ops::fmac(w11, 0.20317460317460317, Ops::fmac(Lam[4], 0.4740740740740741, Ops::mulc(Lam[2], 0.6772486772486772)));
    K[72] = Ops::fmac(w8, -0.5417989417989418, Ops::fmac(Lam[4], -0.8126984126984127, Ops::mulc(Lam[3], 0.8126984126984127)));
    K[73] = Ops::fmac(w32, 5.147089947089947, Ops::mulc(Lam[3], 0.2708994708994709));
    K[74] = Ops::fmac(w33, -1.3544973544973544, Ops::mulc(Lam[3], 0.2708994708994709));
    K[75] = Ops::fmac(w12, 4.1989417989417985, Ops::mulc(Lam[0], 3.657142857142857));
    K[76] = Ops::fmac(Lam[5], -1.5238095238095237, Ops::fmac(Lam[2], 1.0497354497354496, Ops::mulc(Lam[0], -1.3206349206349206)));
    K[77] = Ops::fmac(w10, 0.6772486772486772, Ops::mulc(Lam[2], -0.6772486772486772));
    K[78] = Ops::fmac(w6, 0.20317460317460317, Ops::mulc(Lam[1], 0.40634920634920635));
    K[79] = Ops::fmac(w14, 0.08465608465608465, Ops::fmac(Lam[2], 0.2201058201058201, Ops::mulc(Lam[1], 0.3047619047619048)));
    K[80] = Ops::fmac(w14, 0.20317460317460317, Ops::fmac(Lam[2], 0.4740740740740741, Ops::mulc(Lam[1], 0.6772486772486772)));
    K[81] = Ops::fmac(w23, 5.147089947089947, Ops::mulc(Lam[0], 0.2708994708994709));
    K[82] = Ops::fmac(w24, -1.3544973544973544, Ops::mulc(Lam[0], 0.2708994708994709));
    K[83] = Ops::fmac(w14, -0.5417989417989418, Ops::fmac(Lam[1], -0.8126984126984127, Ops::mulc(Lam[0], 0.8126984126984127)));
    K[84] = Ops::fmac(w10, 4.901587301587302, Ops::mulc(Lam[2], 3.8857142857142857));
    K[85] = Ops::fmac(Lam[5], -1.3206349206349206, Ops::fmac(Lam[2], 1.0497354497354496, Ops::mulc(Lam[0], -1.5238095238095237)));
    K[86] = Ops::fmac(w12, 0.08465608465608465, Ops::fmac(Lam[4], 0.2201058201058201, Ops::mulc(Lam[1], 0.3047619047619048)));
    K[87] = Ops::fmac(w22, -0.7873015873015873, Ops::mulc(Lam[5], -0.2920634920634921));
    K[88] = Ops::fmac(w20, -1.5238095238095237, Ops::fmac(Lam[4], -0.5925925925925926, Ops::mulc(Lam[2], -0.9312169312169312)));
    K[89] = Ops::fmac(w35, 1.8285714285714285, Ops::mulc(Lam[5], -1.0158730158730158));
    K[90] = Ops::fmac(w10, -0.6095238095238096, Ops::fmac(w1, -1.4222222222222223, Ops::mulc(Lam[2], -1.0158730158730158)));
    K[91] = Ops::fmac(w37, 1.8285714285714285, Ops::mulc(Lam[0], -1.0158730158730158));
    K[92] = Ops::fmac(w8, 4.1989417989417985, Ops::mulc(Lam[5], 3.657142857142857));
    K[93] = Ops::fmac(w12, 0.20317460317460317, Ops::fmac(Lam[4], 0.4740740740740741, Ops::mulc(Lam[1], 0.6772486772486772)));
    K[94] = Ops::fmac(w20, -1.5238095238095237, Ops::fmac(Lam[4], -0.9312169312169312, Ops::mulc(Lam[2], -0.5925925925925926)));
    K[95] = Ops::fmac(w22, 4.1989417989417985, Ops::mulc(Lam[5], 1.8285714285714285));
    K[96] = Ops::fmac(w7, -0.5417989417989418, Ops::fmac(Lam[5], 0.8126984126984127, Ops::mulc(Lam[4], -0.8126984126984127)));
    K[97] = Ops::fmac(w33, -1.3544973544973544, Ops::mulc(Lam[5], 0.2708994708994709));
    K[98] = Ops::fmac(w32, 5.147089947089947, Ops::mulc(Lam[5], 0.2708994708994709));
    K[99] = Ops::fmac(w14, 4.1989417989417985, Ops::mulc(Lam[3], 3.657142857142857));
    K[100] = Ops::fmac(Lam[5], -1.5238095238095237, Ops::fmac(Lam[4], 1.0497354497354496, Ops::mulc(Lam[3], -1.3206349206349206)));
    K[101] = Ops::fmac(w13, 0.6772486772486772, Ops::mulc(Lam[4], -0.6772486772486772));
    K[102] = Ops::fmac(w24, -1.3544973544973544, Ops::mulc(Lam[3], 0.2708994708994709));
    K[103] = Ops::fmac(w23, 5.147089947089947, Ops::mulc(Lam[3], 0.2708994708994709));
    K[104] = Ops::fmac(w12, -0.5417989417989418, Ops::fmac(Lam[3], 0.8126984126984127, Ops::mulc(Lam[1], -0.8126984126984127)));
    K[105] = Ops::fmac(w13, 4.901587301587302, Ops::mulc(Lam[4], 3.8857142857142857));
    K[106] = Ops::fmac(Lam[5], -1.3206349206349206, Ops::fmac(Lam[4], 1.0497354497354496, Ops::mulc(Lam[3], -1.5238095238095237)));
    K[107] = Ops::fmac(w13, -0.6095238095238096, Ops::fmac(w0, -1.4222222222222223, Ops::mulc(Lam[4], -1.0158730158730158)));
    K[108] = Ops::fmac(w36, 1.8285714285714285, Ops::mulc(Lam[5], -1.0158730158730158));
    K[109] = Ops::fmac(w37, 1.8285714285714285, Ops::mulc(Lam[3], -1.0158730158730158));
    K[110] = Ops::fmac(w4, 4.1989417989417985, Ops::mulc(Lam[5], 3.657142857142857));
    K[111] = Ops::fmac(w29, -1.3544973544973544, Ops::mulc(Lam[5], 0.2708994708994709));
    K[112] = Ops::fmac(w11, -0.5417989417989418, Ops::fmac(Lam[5], 0.8126984126984127, Ops::mulc(Lam[2], -0.8126984126984127)));
    K[113] = Ops::fmac(w28, 5.147089947089947, Ops::mulc(Lam[5], 0.2708994708994709));
    K[114] = Ops::mulc(w16, 11.377777777777778);
    K[115] = Ops::fmac(w9, -1.6253968253968254, Ops::fmac(w6, 1.6253968253968254, Ops::mulc(Lam[1], 4.876190476190477)));
    K[116] = Ops::fmac(w10, -1.6253968253968254, Ops::fmac(w5, 1.6253968253968254, Ops::mulc(Lam[2], 4.876190476190477)));
    K[117] = Ops::mulc(w16, 11.377777777777778);
    K[118] = Ops::fmac(w13, -1.6253968253968254, Ops::fmac(w3, 1.6253968253968254, Ops::mulc(Lam[4], 4.876190476190477)));
    K[119] = Ops::mulc(w16, 11.377777777777778);
  }
  template <class Ops> __device__ __forceinline__ static void helmholtz_upper(const typename Ops::T* Lam, const typename Ops::T& vol, typename Ops::T* K) {
    const typename Ops::T w0 = Ops::add(Lam[1], Lam[2]);
    const typename Ops::T w1 = Ops::add(Lam[1], Lam[4]);
    const typename Ops::T w2 = Ops::add(Lam[2], Lam[4]);
    const typename Ops::T w3 = Ops::add(Lam[0], w0);
    const typename Ops::T w4 = Ops::add(Lam[3], Lam[4]);
    const typename Ops::T w5 = Ops::add(Lam[3], w1);
    const typename Ops::T w6 = Ops::add(Lam[5], w2);
    const typename Ops::T w7 = Ops::add(Lam[0], Lam[1]);
    const typename Ops::T w8 = Ops::add(Lam[0], Lam[2]);
    const typename Ops::T w9 = Ops::add(Lam[0], Lam[3]);
    const typename Ops::T w10 = Ops::add(Lam[0], Lam[5]);
    const typename Ops::T w11 = Ops::add(Lam[1], Lam[3]);
    const typename Ops::T w12 = Ops::add(Lam[2], Lam[5]);
    const typename Ops::T w13 = Ops::add(Lam[3], Lam[5]);
    const typename Ops::T w14 = Ops::add(Lam[4], Lam[5]);
    const typename Ops::T w15 = Ops::add(Lam[5], w3);
    const typename Ops::T w16 = Ops::add(w4, w15);
    const typename Ops::T w17 = Ops::fmac(Lam[4], 2.0930232558139537, Lam[0]);
    const typename Ops::T w18 = Ops::fmac(Lam[4], 1.7692307692307692, Lam[0]);
    const typename Ops::T w19 = Ops::fmac(w0, 0.2, Lam[0]);
    const typename Ops::T w20 = Ops::fmac(Lam[5], 0.4777777777777778, Lam[1]);
    const typename Ops::T w21 = Ops::fmac(Lam[5], 0.5652173913043478, Lam[1]);
    const typename Ops::T w22 = Ops::fmac(w2, 0.5, Lam[1]);
    const typename Ops::T w23 = Ops::fmac(w6, 0.631578947368421, Lam[1]);
    const typename Ops::T w24 = Ops::fmac(w6, 0.4, Lam[1]);
    const typename Ops::T w25 = Ops::fmac(Lam[3], 0.4777777777777778, Lam[2]);
    const typename Ops::T w26 = Ops::fmac(Lam[3], 0.5652173913043478, Lam[2]);
    const typename Ops::T w27 = Ops::fmac(w1, 0.5, Lam[2]);
    const typename Ops::T w28 = Ops::fmac(w5, 0.631578947368421, Lam[2]);
    const typename Ops::T w29 = Ops::fmac(w5, 0.4, Lam[2]);
    const typename Ops::T w30 = Ops::fmac(w1, 0.2, Lam[3]);
    const typename Ops::T w31 = Ops::fmac(w0, 0.5, Lam[4]);
    const typename Ops::T w32 = Ops::fmac(w3, 0.631578947368421, Lam[4]);
    const typename Ops::T w33 = Ops::fmac(w3, 0.4, Lam[4]);
    const typename Ops::T w34 = Ops::fmac(w2, 0.2, Lam[5]);
    const typename Ops::T w35 = Ops::fmac(w18, 1.4444444444444444, w0);
    const typename Ops::T w36 = Ops::fmac(w26, 2.5555555555555554, w1);
    const typename Ops::T w37 = Ops::fmac(w21, 2.5555555555555554, w2);
    const typename Ops::T m0 = Ops::mulc(vol, 0.0051146384479717815);
    const typename Ops::T m1 = Ops::mulc(vol, -0.0004761904761904762);
    const typename Ops::T m2 = Ops::mulc(vol, 0.0028218694885361554);
    const typename Ops::T m3 = Ops::mulc(vol, -0.0014109347442680777);
    const typename Ops::T m4 = Ops::mulc(vol, -0.0019753086419753087);
    const typename Ops::T m5 = Ops::mulc(vol, -0.00021164021164021165);
    const typename Ops::T m6 = Ops::mulc(vol, -0.0028218694885361554);
    const typename Ops::T m7 = Ops::mulc(vol, 0.045149911816578486);
    const typename Ops::T m8 = Ops::mulc(vol, -0.022574955908289243);
    const typename Ops::T m9 = Ops::mulc(vol, 0.013544973544973546);
    const typename Ops::T m10 = Ops::mulc(vol, 0.022574955908289243);
    const typename Ops::T m11 = Ops::mulc(vol, -0.016931216931216932);
    const typename Ops::T m12 = Ops::mulc(vol, 0.009029982363315696);
    const typename Ops::T m13 = Ops::mulc(vol, 0.001128747795414462);
    const typename Ops::T m14 = Ops::mulc(vol, 0.004514991181657848);
    const typename Ops::T m15 = Ops::mulc(vol, -0.004514991181657848);
    const typename Ops::T m16 = Ops::mulc(vol, 0.05587301587301587);
    const typename Ops::T m17 = Ops::mulc(vol, 0.0008465608465608466);
    const typename Ops::T m18 = Ops::mulc(vol, 0.006772486772486773);
    const typename Ops::T m19 = Ops::mulc(vol, -0.013544973544973546);
    const typename Ops::T m20 = Ops::mulc(vol, 0.18962962962962962);
    const typename Ops::T m21 = Ops::mulc(vol, -0.02708994708994709);
    K[0] = Ops::fmac(Lam[0], 0.746031746031746, m0);
    K[1] = Ops::fmac(Lam[1], -0.11322751322751323, m1);
    K[2] = Ops::fmac(Lam[2], -0.11322751322751323, m1);
    K[3] = Ops::fmac(Lam[1], 1.5576719576719578, Ops::fmac(Lam[0], 0.25396825396825395, m2));
    K[4] = Ops::fmac(Lam[1], -0.8507936507936508, Ops::fmac(Lam[0], 0.08465608465608465, m3));
    K[5] = Ops::fmac(Lam[1], 0.40634920634920635, Ops::mulc(Lam[0], -0.08465608465608465));
    K[6] = Ops::fmac(Lam[2], 1.5576719576719578, Ops::fmac(Lam[0], 0.25396825396825395, m2));
    K[7] = Ops::fmac(Lam[2], -0.8507936507936508, Ops::fmac(Lam[0], 0.08465608465608465, m3));
    K[8] = Ops::fmac(Lam[2], 0.40634920634920635, Ops::mulc(Lam[0], -0.08465608465608465));
    K[9] = Ops::fmac(w0, -0.08465608465608465, m4);
    K[10] = Ops::fmac(w0, -0.08465608465608465, m5);
    K[11] = Ops::fmac(w0, -0.08465608465608465, m4);
    K[12] = Ops::fmac(w0, 0.6349206349206349, Ops::fmac(Lam[0], 0.4656084656084656, m2));
    K[13] = Ops::fmac(w19, -0.21164021164021163, m6);
    K[14] = Ops::fmac(w19, -0.21164021164021163, m6);
    K[15] = Ops::fmac(Lam[3], 0.746031746031746, m0);
    K[16] = Ops::fmac(Lam[4], -0.11322751322751323, m1);
    K[17] = Ops::fmac(Lam[3], -0.08465608465608465, Ops::mulc(Lam[1], 0.40634920634920635));
    K[18] = Ops::fmac(Lam[3], 0.08465608465608465, Ops::fmac(Lam[1], -0.8507936507936508, m3));
    K[19] = Ops::fmac(Lam[3], 0.25396825396825395, Ops::fmac(Lam[1], 1.5576719576719578, m2));
    K[20] = Ops::fmac(w1, -0.08465608465608465, m4);
    K[21] = Ops::fmac(w1, -0.08465608465608465, m5);
    K[22] = Ops::fmac(w1, -0.08465608465608465, m4);
    K[23] = Ops::fmac(Lam[4], 1.5576719576719578, Ops::fmac(Lam[3], 0.25396825396825395, m2));
    K[24] = Ops::fmac(Lam[4], -0.8507936507936508, Ops::fmac(Lam[3], 0.08465608465608465, m3));
    K[25] = Ops::fmac(Lam[4], 0.40634920634920635, Ops::mulc(Lam[3], -0.08465608465608465));
    K[26] = Ops::fmac(w30, -0.21164021164021163, m6);
    K[27] = Ops::fmac(w1, 0.6349206349206349, Ops::fmac(Lam[3], 0.4656084656084656, m2));
    K[28] = Ops::fmac(w30, -0.21164021164021163, m6);
    K[29] = Ops::fmac(Lam[5], 0.746031746031746, m0);
    K[30] = Ops::fmac(w2, -0.08465608465608465, m4);
    K[31] = Ops::fmac(w2, -0.08465608465608465, m5);
    K[32] = Ops::fmac(w2, -0.08465608465608465, m4);
    K[33] = Ops::fmac(Lam[5], -0.08465608465608465, Ops::mulc(Lam[2], 0.40634920634920635));
    K[34] = Ops::fmac(Lam[5], 0.08465608465608465, Ops::fmac(Lam[2], -0.8507936507936508, m3));
    K[35] = Ops::fmac(Lam[5], 0.25396825396825395, Ops::fmac(Lam[2], 1.5576719576719578, m2));
    K[36] = Ops::fmac(Lam[5], -0.08465608465608465, Ops::mulc(Lam[4], 0.40634920634920635));
    K[37] = Ops::fmac(Lam[5], 0.08465608465608465, Ops::fmac(Lam[4], -0.8507936507936508, m3));
    K[38] = Ops::fmac(Lam[5], 0.25396825396825395, Ops::fmac(Lam[4], 1.5576719576719578, m2));
    K[39] = Ops::fmac(w34, -0.21164021164021163, m6);
    K[40] = Ops::fmac(w34, -0.21164021164021163, m6);
    K[41] = Ops::fmac(w2, 0.6349206349206349, Ops::fmac(Lam[5], 0.4656084656084656, m2));
    K[42] = Ops::fmac(w11, 4.1989417989417985, Ops::fmac(Lam[0], 3.657142857142857, m7));
    K[43] = Ops::fmac(Lam[3], -1.5238095238095237, Ops::fmac(Lam[1], 1.0497354497354496, Ops::fmac(Lam[0], -1.3206349206349206, m8)));
    K[44] = Ops::fmac(w9, 0.6772486772486772, Ops::fmac(Lam[1], -0.6772486772486772, m9));
    K[45] = Ops::fmac(w31, 4.1989417989417985, Ops::fmac(Lam[0], 1.8285714285714285, m10));
    K[46] = Ops::fmac(w17, -0.728042328042328, Ops::fmac(Lam[2], -0.9312169312169312, Ops::fmac(Lam[1], -0.5925925925925926, m11)));
    K[47] = Ops::fmac(w7, 0.20317460317460317, Ops::fmac(Lam[4], 0.6772486772486772, Ops::fmac(Lam[2], 0.4740740740740741, m12)));
    K[48] = Ops::fmac(w4, 0.20317460317460317, Ops::fmac(Lam[2], 0.6772486772486772, Ops::fmac(Lam[1], 0.4740740740740741, m12)));
    K[49] = Ops::fmac(w4, 0.08465608465608465, Ops::fmac(Lam[2], 0.3047619047619048, Ops::fmac(Lam[1], 0.2201058201058201, m13)));
    K[50] = Ops::fmac(w5, 0.20317460317460317, Ops::fmac(Lam[2], 0.40634920634920635, m14));
    K[51] = Ops::fmac(w28, 5.147089947089947, Ops::fmac(Lam[0], 0.2708994708994709, m10));
    K[52] = Ops::fmac(w4, -0.5417989417989418, Ops::fmac(Lam[2], -0.8126984126984127, Ops::fmac(Lam[0], 0.8126984126984127, m14)));
    K[53] = Ops::fmac(w29, -1.3544973544973544, Ops::fmac(Lam[0], 0.2708994708994709, m15));
    K[54] = Ops::fmac(w9, 4.901587301587302, Ops::fmac(Lam[1], 3.8857142857142857, m16));
    K[55] = Ops::fmac(Lam[3], -1.3206349206349206, Ops::fmac(Lam[1], 1.0497354497354496, Ops::fmac(Lam[0], -1.5238095238095237, m8)));
    K[56] = Ops::fmac(w17, -0.728042328042328, Ops::fmac(Lam[2], -0.5925925925925926, Ops::fmac(Lam[1], -0.9312169312169312, m11)));
    K[57] = Ops::fmac(w31, -0.7873015873015873, Ops::fmac(Lam[0], -0.2920634920634921, m17));
    K[58] = Ops::fmac(w7, 0.08465608465608465, Ops::fmac(Lam[4], 0.3047619047619048, Ops::fmac(Lam[2], 0.2201058201058201, m13)));
    K[59] = Ops::fmac(w25, -1.5238095238095237, Ops::fmac(Lam[4], -0.5925925925925926, Ops::fmac(Lam[1], -0.9312169312169312, m11)));
    K[60] = Ops::fmac(w27, -0.7873015873015873, Ops::fmac(Lam[3], -0.2920634920634921, m17));
    K[61] = Ops::fmac(w11, 0.08465608465608465, Ops::fmac(Lam[4], 0.2201058201058201, Ops::fmac(Lam[2], 0.3047619047619048, m13)));
    K[62] = Ops::fmac(w35, 1.8285714285714285, Ops::fmac(Lam[3], -1.0158730158730158, m18));
    K[63] = Ops::fmac(w36, 1.8285714285714285, Ops::fmac(Lam[0], -1.0158730158730158, m18));
    K[64] = Ops::fmac(w9, -0.6095238095238096, Ops::fmac(w2, -1.4222222222222223, Ops::fmac(Lam[1], -1.0158730158730158, m19)));
    K[65] = Ops::fmac(w7, 4.1989417989417985, Ops::fmac(Lam[3], 3.657142857142857, m7));
    K[66] = Ops::fmac(w8, 0.20317460317460317, Ops::fmac(Lam[4], 0.6772486772486772, Ops::fmac(Lam[1], 0.4740740740740741, m12)));
    K[67] = Ops::fmac(w8, 0.08465608465608465, Ops::fmac(Lam[4], 0.3047619047619048, Ops::fmac(Lam[1], 0.2201058201058201, m13)));
    K[68] = Ops::fmac(w3, 0.20317460317460317, Ops::fmac(Lam[4], 0.40634920634920635, m14));
    K[69] = Ops::fmac(w27, 4.1989417989417985, Ops::fmac(Lam[3], 1.8285714285714285, m10));
    K[70] = Ops::fmac(w25, -1.5238095238095237, Ops::fmac(Lam[4], -0.9312169312169312, Ops::fmac(Lam[1], -0.5925925925925926, m11)));
    K[71] = Ops::fmac(w11, 0.20317460317460317, Ops::fmac(Lam[4], 0.4740740740740741, Ops::fmac(Lam[2], 0.6772486772486772, m12)));
    K[72] = Ops::fmac(w8, -0.5417989417989418, Ops::fmac(Lam[4], -0.8126984126984127, Ops::fmac(Lam[3], 0.8126984126984127, m14)));
    K[73] = Ops::fmac(w32, 5.147089947089947, Ops::fmac(Lam[3], 0.2708994708994709, m10));
    K[74] = Ops::fmac(w33, -1.3544973544973544, Ops::fmac(Lam[3], 0.2708994708994709, m15));
    K[75] = Ops::fmac(w12, 4.1989417989417985, Ops::fmac(Lam[0], 3.657142857142857, m7));
    K[76] = Ops::fmac(Lam[5], -1.5238095238095237, Ops::fmac(Lam[2], 1.0497354497354496, Ops::fmac(Lam[0], -1.3206349206349206, m8)));
    K[77] = Ops::fmac(w10, 0.6772486772486772, Ops::fmac(Lam[2], -0.6772486772486772, m9));
    K[78] = Ops::fmac(w6, 0.20317460317460317, Ops::fmac(Lam[1], 0.40634920634920635, m14));
    K[79] = Ops::fmac(w14, 0.08465608465608465, Ops::fmac(Lam[2], 0.2201058201058201, Ops::fmac(Lam[1], 0.3047619047619048, m13)));
    K[80] = Ops::fmac(w14, 0.20317460317460317, Ops::fmac(Lam[2], 0.4740740740740741, Ops::fmac(Lam[1], 0.6772486772486772, m12)));
    K[81] = Ops::fmac(w23, 5.147089947089947, Ops::fmac(Lam[0], 0.2708994708994709, m10));
    K[82] = Ops::fmac(w24, -1.3544973544973544, Ops::fmac(Lam[0], 0.2708994708994709, m15));
    K[83] = Ops::fmac(w14, -0.5417989417989418, Ops::fmac(Lam[1], -0.8126984126984127, Ops::fmac(Lam[0], 0.8126984126984127, m14)));
    K[84] = Ops::fmac(w10, 4.901587301587302, Ops::fmac(Lam[2], 3.8857142857142857, m16));
    K[85] = Ops::fmac(Lam[5], -1.3206349206349206, Ops::fmac(Lam[2], 1.0497354497354496, Ops::fmac(Lam[0], -1.5238095238095237, m8)));
    K[86] = Ops::fmac(w12, 0.08465608465608465, Ops::fmac(Lam[4], 0.2201058201058201, Ops::fmac(Lam[1], 0.3047619047619048, m13)));
    K[87] = Ops::fmac(w22, -0.7873015873015873, Ops::fmac(Lam[5], -0.2920634920634921, m17));
    K[88] = Ops::fmac(w20, -1.5238095238095237, Ops::fmac(Lam[4], -0.5925925925925926, Ops::fmac(Lam[2], -0.9312169312169312, m11)));
    K[89] = Ops::fmac(w35, 1.8285714285714285, Ops::fmac(Lam[5], -1.0158730158730158, m18));
    K[90] = Ops::fmac(w10, -0.6095238095238096, Ops::fmac(w1, -1.4222222222222223, Ops::fmac(Lam[2], -1.0158730158730158, m19)));
    K[91] = Ops::fmac(w37, 1.8285714285714285, Ops::fmac(Lam[0], -1.0158730158730158, m18));
    K[92] = Ops::fmac(w8, 4.1989417989417985, Ops::fmac(Lam[5], 3.657142857142857, m7));
    K[93] = Ops::fmac(w12, 0.20317460317460317, Ops::fmac(Lam[4], 0.4740740740740741, Ops::fmac(Lam[1], 0.6772486772486772, m12)));
    K[94] = Ops::fmac(w20, -1.5238095238095237, Ops::fmac(Lam[4], -0.9312169312169312, Ops::fmac(Lam[2], -0.5925925925925926, m11)));
    K[95] = Ops::fmac(w22, 4.1989417989417985, Ops::fmac(Lam[5], 1.8285714285714285, m10));
    K[96] = Ops::fmac(w7, -0.5417989417989418, Ops::fmac(Lam[5], 0.8126984126984127, Ops::fmac(Lam[4], -0.8126984126984127, m14)));
    K[97] = Ops::fmac(w33, -1.3544973544973544, Ops::fmac(Lam[5], 0.2708994708994709, m15));
    K[98] = Ops::fmac(w32, 5.147089947089947, Ops::fmac(Lam[5], 0.2708994708994709, m10));
    K[99] = Ops::fmac(w14, 4.1989417989417985, Ops::fmac(Lam[3], 3.657142857142857, m7));
    K[100] = Ops::fmac(Lam[5], -1.5238095238095237, Ops::fmac(Lam[4], 1.0497354497354496, Ops::fmac(Lam[3], -1.3206349206349206, m8)));
    K[101] = Ops::fmac(w13, 0.6772486772486772, Ops::fmac(Lam[4], -0.6772486772486772, m9));
    K[102] = Ops::fmac(w24, -1.3544973544973544, Ops::fmac(Lam[3], 0.2708994708994709, m15));
    K[103] = Ops::fmac(w23, 5.147089947089947, Ops::fmac(Lam[3], 0.2708994708994709, m10));
    K[104] = Ops::fmac(w12, -0.5417989417989418, Ops::fmac(Lam[3], 0.8126984126984127, Ops::fmac(Lam[1], -0.8126984126984127, m14)));
    K[105] = Ops::fmac(w13, 4.901587301587302, Ops::fmac(Lam[4], 3.8857142857142857, m16));
    K[106] = Ops::fmac(Lam[5], -1.3206349206349206, Ops::fmac(Lam[4], 1.0497354497354496, Ops::fmac(Lam[3], -1.5238095238095237, m8)));
    K[107] = Ops::fmac(w13, -0.6095238095238096, Ops::fmac(w0, -1.4222222222222223, Ops::fmac(Lam[4], -1.0158730158730158, m19)));
    K[108] = Ops::fmac(w36, 1.8285714285714285, Ops::fmac(Lam[5], -1.0158730158730158, m18));
    K[109] = Ops::fmac(w37, 1.8285714285714285, Ops::fmac(Lam[3], -1.0158730158730158, m18));
    K[110] = Ops::fmac(w4, 4.1989417989417985, Ops::fmac(Lam[5], 3.657142857142857, m7));
    K[111] = Ops::fmac(w29, -1.3544973544973544, Ops::fmac(Lam[5], 0.2708994708994709, m15));
    K[112] = Ops::fmac(w11, -0.5417989417989418, Ops::fmac(Lam[5], 0.8126984126984127, Ops::fmac(Lam[2], -0.8126984126984127, m14)));
    K[113] = Ops::fmac(w28, 5.147089947089947, Ops::fmac(Lam[5], 0.2708994708994709, m10));
    K[114] = Ops::fmac(w16, 11.377777777777778, m20);
    K[115] = Ops::fmac(w9, -1.6253968253968254, Ops::fmac(w6, 1.6253968253968254, Ops::fmac(Lam[1], 4.876190476190477, m21)));
    K[116] = Ops::fmac(w10, -1.6253968253968254, Ops::fmac(w5, 1.6253968253968254, Ops::fmac(Lam[2], 4.876190476190477, m21)));
    K[117] = Ops::fmac(w16, 11.377777777777778, m20);
    K[118] = Ops::fmac(w13, -1.6253968253968254, Ops::fmac(w3, 1.6253968253968254, Ops::fmac(Lam[4], 4.876190476190477, m21)));
    K[119] = Ops::fmac(w16, 11.377777777777778, m20);
  }
  template <class Ops> __device__ __forceinline__ static void mass_upper(const typename Ops::T& vol, typename Ops::T* K) {
    const typename Ops::T m0 = Ops::mulc(vol, 0.0051146384479717815);
    const typename Ops::T m1 = Ops::mulc(vol, -0.0004761904761904762);
    const typename Ops::T m2 = Ops::mulc(vol, 0.0028218694885361554);
    const typename Ops::T m3 = Ops::mulc(vol, -0.0014109347442680777);
    const typename Ops::T m4 = Ops::mulc(vol, -0.0019753086419753087);
    const typename Ops::T m5 = Ops::mulc(vol, -0.00021164021164021165);
    const typename Ops::T m6 = Ops::mulc(vol, -0.0028218694885361554);
    const typename Ops::T m7 = Ops::mulc(vol, 0.045149911816578486);
    const typename Ops::T m8 = Ops::mulc(vol, -0.022574955908289243);
    const typename Ops::T m9 = Ops::mulc(vol, 0.013544973544973546);
    const typename Ops::T m10 = Ops::mulc(vol, 0.022574955908289243);
    const typename Ops::T m11 = Ops::mulc(vol, -0.016931216931216932);
    const typename Ops::T m12 = Ops::mulc(vol, 0.009029982363315696);
    const typename Ops::T m13 = Ops::mulc(vol, 0.001128747795414462);
    const typename Ops::T m14 = Ops::mulc(vol, 0.004514991181657848);
    const typename Ops::T m15 = Ops::mulc(vol, -0.004514991181657848);
    const typename Ops::T m16 = Ops::mulc(vol, 0.05587301587301587);
    const typename Ops::T m17 = Ops::mulc(vol, 0.0008465608465608466);
    const typename Ops::T m18 = Ops::mulc(vol, 0.006772486772486773);
    const typename Ops::T m19 = Ops::mulc(vol, -0.013544973544973546);
    const typename Ops::T m20 = Ops::mulc(vol, 0.18962962962962962);
    const typename Ops::T m21 = Ops::mulc(vol, -0.02708994708994709);
    K[0] = m0;
    K[1] = m1;
    K[2] = m1;
    K[3] = m2;
    K[4] = m3;
    K[5] = Ops::zero();
    K[6] = m2;
    K[7] = m3;
    K[8] = Ops::zero();
    K[9] = m4;
    K[10] = m5;
    K[11] = m4;
    K[12] = m2;
    K[13] = m6;
    K[14] = m6;
    K[15] = m0;
    K[16] = m1;
    K[17] = Ops::zero();
    K[18] = m3;
    K[19] = m2;
    K[20] = m4;
    K[21] = m5;
    K[22] = m4;
    K[23] = m2;
    K[24] = m3;
    K[25] = Ops::zero();
    K[26] = m6;
    K[27] = m2;
    K[28] = m6;
    K[29] = m0;
    K[30] = m4;
    K[31] = m5;
    K[32] = m4;
    K[33] = Ops::zero();
    K[34] = m3;
    K[35] = m2;
    K[36] = Ops::zero();
    K[37] = m3;
    K[38] = m2;
    K[39] = m6;
    K[40] = m6;
    K[41] = m2;
    K[42] = m7;
    K[43] = m8;
    K[44] = m9;
    K[45] = m10;
    K[46] = m11;
    K[47] = m12;
    K[48] = m12;
    K[49] = m13;
    K[50] = m14;
    K[51] = m10;
    K[52] = m14;
    K[53] = m15;
    K[54] = m16;
    K[55] = m8;
    K[56] = m11;
    K[57] = m17;
    K[58] = m13;
    K[59] = m11;
    K[60] = m17;
    K[61] = m13;
    K[62] = m18;
    K[63] = m18;
    K[64] = m19;
    K[65] = m7;
    K[66] = m12;
    K[67] = m13;
    K[68] = m14;
    K[69] = m10;
    K[70] = m11;
    K[71] = m12;
    K[72] = m14;
    K[73] = m10;
    K[74] = m15;
    K[75] = m7;
    K[76] = m8;
    K[77] = m9;
    K[78] = m14;
    K[79] = m13;
    K[80] = m12;
    K[81] = m10;
    K[82] = m15;
    K[83] = m14;
    K[84] = m16;
    K[85] = m8;
    K[86] = m13;
    K[87] = m17;
    K[88] = m11;
    K[89] = m18;
    K[90] = m19;
    K[91] = m18;
    K[92] = m7;
    K[93] = m12;
    K[94] = m11;
    K[95] = m10;
    K[96] = m14;
    K[97] = m15;
    K[98] = m10;
    K[99] = m7;
    K[100] = m8;
    K[101] = m9;
    K[102] = m15;
    K[103] = m10;
    K[104] = m14;
    K[105] = m16;
    K[106] = m8;
    K[107] = m19;
    K[108] = m18;
    K[109] = m18;
    K[110] = m7;
    K[111] = m15;
    K[112] = m14;
    K[113] = m10;
    K[114] = m20;
    K[115] = m21;
    K[116] = m21;
    K[117] = m20;
    K[118] = m21;
    K[119] = m20;
  }
  template <class Ops, bool STIFF, bool MASS> __device__ __forceinline__ static void action_upper(const typename Ops::T* Lam, const typename Ops::T& vol, const typename Ops::T* x, typename Ops::T* y) {
    typename Ops::T k;
    if constexpr (STIFF && MASS) {
      const typename Ops::T w0 = Ops::add(Lam[1], Lam[2]);
      const typename Ops::T w1 = Ops::add(Lam[1], Lam[4]);
      const typename Ops::T w2 = Ops::add(Lam[2], Lam[4]);
      const typename Ops::T w3 = Ops::add(Lam[0], w0);
      const typename Ops::T w4 = Ops::add(Lam[3], Lam[4]);
      const typename Ops::T w5 = Ops::add(Lam[3], w1);
      const typename Ops::T w6 = Ops::add(Lam[5], w2);
      const typename Ops::T w7 = Ops::add(Lam[0], Lam[1]);
      const typename Ops::T w8 = Ops::add(Lam[0], Lam[2]);
      const typename Ops::T w9 = Ops::add(Lam[0], Lam[3]);
      const typename Ops::T w10 = Ops::add(Lam[0], Lam[5]);
      const typename Ops::T w11 = Ops::add(Lam[1], Lam[3]);
      const typename Ops::T w12 = Ops::add(Lam[2], Lam[5]);
      const typename Ops::T w13 = Ops::add(Lam[3], Lam[5]);
      const typename Ops::T w14 = Ops::add(Lam[4], Lam[5]);
      const typename Ops::T w15 = Ops::add(Lam[5], w3);
      const typename Ops::T w16 = Ops::add(w4, w15);
      const typename Ops::T w17 = Ops::fmac(Lam[4], 2.0930232558139537, Lam[0]);
      const typename Ops::T w18 = Ops::fmac(Lam[4], 1.7692307692307692, Lam[0]);
      const typename Ops::T w19 = Ops::fmac(w0, 0.2, Lam[0]);
      const typename Ops::T w20 = Ops::fmac(Lam[5], 0.4777777777777778, Lam[1]);
      const typename Ops::T w21 = Ops::fmac(Lam[5], 0.5652173913043478, Lam[1]);
      const typename Ops::T w22 = Ops::fmac(w2, 0.5, Lam[1]);
      const typename Ops::T w23 = Ops::fmac(w6, 0.631578947368421, Lam[1]);
      const typename Ops::T w24 = Ops::fmac(w6, 0.4, Lam[1]);
      const typename Ops::T w25 = Ops::fmac(Lam[3], 0.4777777777777778, Lam[2]);
      const typename Ops::T w26 = Ops::fmac(Lam[3], 0.5652173913043478, Lam[2]);
      const typename Ops::T w27 = Ops::fmac(w1, 0.5, Lam[2]);
      const typename Ops::T w28 = Ops::fmac(w5, 0.631578947368421, Lam[2]);
      const typename Ops::T w29 = Ops::fmac(w5, 0.4, Lam[2]);
      const typename Ops::T w30 = Ops::fmac(w1, 0.2, Lam[3]);
      const typename Ops::T w31 = Ops::fmac(w0, 0.5, Lam[4]);
      const typename Ops::T w32 = Ops::fmac(w3, 0.631578947368421, Lam[4]);
      const typename Ops::T w33 = Ops::fmac(w3, 0.4, Lam[4]);
      const typename Ops::T w34 = Ops::fmac(w2, 0.2, Lam[5]);
      const typename Ops::T w35 = Ops::fmac(w18, 1.4444444444444444, w0);
      const typename Ops::T w36 = Ops::fmac(w26, 2.5555555555555554, w1);
      const typename Ops::T w37 = Ops::fmac(w21, 2.5555555555555554, w2);
      const typename Ops::T m0 = Ops::mulc(vol, 0.0051146384479717815);
      const typename Ops::T m1 = Ops::mulc(vol, -0.0004761904761904762);
      const typename Ops::T m2 = Ops::mulc(vol, 0.0028218694885361554);
      const typename Ops::T m3 = Ops::mulc(vol, -0.0014109347442680777);
      const typename Ops::T m4 = Ops::mulc(vol, -0.0019753086419753087);
      const typename Ops::T m5 = Ops::mulc(vol, -0.00021164021164021165);
      const typename Ops::T m6 = Ops::mulc(vol, -0.0028218694885361554);
      const typename Ops::T m7 = Ops::mulc(vol, 0.045149911816578486);
      const typename Ops::T m8 = Ops::mulc(vol, -0.022574955908289243);
      const typename Ops::T m9 = Ops::mulc(vol, 0.013544973544973546);
      const typename Ops::T m10 = Ops::mulc(vol, 0.022574955908289243);
      const typename Ops::T m11 = Ops::mulc(vol, -0.016931216931216932);
      const typename Ops::T m12 = Ops::mulc(vol, 0.009029982363315696);
      const typename Ops::T m13 = Ops::mulc(vol, 0.001128747795414462);
      const typename Ops::T m14 = Ops::mulc(vol, 0.004514991181657848);
      const typename Ops::T m15 = Ops::mulc(vol, -0.004514991181657848);
      const typename Ops::T m16 = Ops::mulc(vol, 0.05587301587301587);
      const typename Ops::T m17 = Ops::mulc(vol, 0.0008465608465608466);
      const typename Ops::T m18 = Ops::mulc(vol, 0.006772486772486773);
      const typename Ops::T m19 = Ops::mulc(vol, -0.013544973544973546);
      const typename Ops::T m20 = Ops::mulc(vol, 0.18962962962962962);
      const typename Ops::T m21 = Ops::mulc(vol, -0.02708994708994709);
      { k = Ops::fmac(Lam[0], 0.746031746031746, m0); y[0] = Ops::mul(k, x[0]); }
      { k = Ops::fmac(Lam[1], -0.11322751322751323, m1); y[0] = Ops::fma3(k, x[1], y[0]); y[1] = Ops::mul(k, x[0]); }
      { k = Ops::fmac(Lam[2], -0.11322751322751323, m1); y[0] = Ops::fma3(k, x[2], y[0]); y[2] = Ops::mul(k, x[0]); }
      { k = Ops::fmac(Lam[1], 1.5576719576719578, Ops::fmac(Lam[0], 0.25396825396825395, m2)); y[0] = Ops::fma3(k, x[3], y[0]); y[3] = Ops::mul(k, x[0]); }
      { k = Ops::fmac(Lam[1], -0.8507936507936508, Ops::fmac(Lam[0], 0.08465608465608465, m3)); y[0] = Ops::fma3(k, x[4], y[0]); y[4] = Ops::mul(k, x[0]); }
      { k = Ops::fmac(Lam[1], 0.40634920634920635, Ops::mulc(Lam[0], -0.08465608465608465)); y[0] = Ops::fma3(k, x[5], y[0]); y[5] = Ops::mul(k, x[0]); }
      { k = Ops::fmac(Lam[2], 1.5576719576719578, Ops::fmac(Lam[0], 0.25396825396825395, m2)); y[0] = Ops::fma3(k, x[6], y[0]); y[6] = Ops::mul(k, x[0]); }
      { k = Ops::fmac(Lam[2], -0.8507936507936508, Ops::fmac(Lam[0], 0.08465608465608465, m3)); y[0] = Ops::fma3(k, x[7], y[0]); y[7] = Ops::mul(k, x[0]); }
      { k = Ops::fmac(Lam[2], 0.40634920634920635, Ops::mulc(Lam[0], -0.08465608465608465)); y[0] = Ops::fma3(k, x[8], y[0]); y[8] = Ops::mul(k, x[0]); }
      { k = Ops::fmac(w0, -0.08465608465608465, m4); y[0] = Ops::fma3(k, x[9], y[0]); y[9] = Ops::mul(k, x[0]); }
      { k = Ops::fmac(w0, -0.08465608465608465, m5); y[0] = Ops::fma3(k, x[10], y[0]); y[10] = Ops::mul(k, x[0]); }
      { k = Ops::fmac(w0, -0.08465608465608465, m4); y[0] = Ops::fma3(k, x[11], y[0]); y[11] = Ops::mul(k, x[0]); }
      { k = Ops::fmac(w0, 0.6349206349206349, Ops::fmac(Lam[0], 0.4656084656084656, m2)); y[0] = Ops::fma3(k, x[12], y[0]); y[12] = Ops::mul(k, x[0]); }
      { k = Ops::fmac(w19, -0.21164021164021163, m6); y[0] = Ops::fma3(k, x[13], y[0]); y[13] = Ops::mul(k, x[0]); }
      { k = Ops::fmac(w19, -0.21164021164021163, m6); y[0] = Ops::fma3(k, x[14], y[0]); y[14] = Ops::mul(k, x[0]); }
      { k = Ops::fmac(Lam[3], 0.746031746031746, m0); y[1] = Ops::fma3(k, x[1], y[1]); }
      { k = Ops::fmac(Lam[4], -0.11322751322751323, m1); y[1] = Ops::fma3(k, x[2], y[1]); y[2] = Ops::fma3(k, x[1], y[2]); }
      { k = Ops::fmac(Lam[3], -0.08465608465608465, Ops::mulc(Lam[1], 0.40634920634920635)); y[1] = Ops::fma3(k, x[3], y[1]); y[3] = Ops::fma3(k, x[1], y[3]); }
      { k = Ops::fmac(Lam[3], 0.08465608465608465, Ops::fmac(Lam[1], -0.8507936507936508, m3)); y[1] = Ops::fma3(k, x[4], y[1]); y[4] = Ops::fma3(k, x[1], y[4]); }
      { k = Ops::fmac(Lam[3], 0.25396825396825395, Ops::fmac(Lam[1], 1.5576719576719578, m2)); y[1] = Ops::fma3(k, x[5], y[1]); y[5] = Ops::fma3(k, x[1], y[5]); }
      { k = Ops::fmac(w1, -0.08465608465608465, m4); y[1] = Ops::fma3(k, x[6], y[1]); y[6] = Ops::fma3(k, x[1], y[6]); }
      { k = Ops::fmac(w1, -0.08465608465608465, m5); y[1] = Ops::fma3(k, x[7], y[1]); y[7] = Ops::fma3(k, x[1], y[7]); }
      { k = Ops::fmac(w1, -0.08465608465608465, m4); y[1] = Ops::fma3(k, x[8], y[1]); y[8] = Ops::fma3(k, x[1], y[8]); }
      { k = Ops::fmac(Lam[4], 1.5576719576719578, Ops::fmac(Lam[3], 0.25396825396825395, m2)); y[1] = Ops::fma3(k, x[9], y[1]); y[9] = Ops::fma3(k, x[1], y[9]); }
      { k = Ops::fmac(Lam[4], -0.8507936507936508, Ops::fmac(Lam[3], 0.08465608465608465, m3)); y[1] = Ops::fma3(k, x[10], y[1]); y[10] = Ops::fma3(k, x[1], y[10]); }
      { k = Ops::fmac(Lam[4], 0.40634920634920635, Ops::mulc(Lam[3], -0.08465608465608465)); y[1] = Ops::fma3(k, x[11], y[1]); y[11] = Ops::fma3(k, x[1], y[11]); }
      { k = Ops::fmac(w30, -0.21164021164021163, m6); y[1] = Ops::fma3(k, x[12], y[1]); y[12] = Ops::fma3(k, x[1], y[12]); }
      { k = Ops::fmac(w1, 0.6349206349206349, Ops::fmac(Lam[3], 0.4656084656084656, m2)); y[1] = Ops::fma3(k, x[13], y[1]); y[13] = Ops::fma3(k, x[1], y[13]); }
      { k = Ops::fmac(w30, -0.21164021164021163, m6); y[1] = Ops::fma3(k, x[14], y[1]); y[14] = Ops::fma3(k, x[1], y[14]); }
      { k = Ops::fmac(Lam[5], 0.746031746031746, m0); y[2] = Ops::fma3(k, x[2], y[2]); }
      { k = Ops::fmac(w2, -0.08465608465608465, m4); y[2] = Ops::fma3(k, x[3], y[2]); y[3] = Ops::fma3(k, x[2], y[3]); }
      { k = Ops::fmac(w2, -0.08465608465608465, m5); y[2] = Ops::fma3(k, x[4], y[2]); y[4] = Ops::fma3(k, x[2], y[4]); }
      { k = Ops::fmac(w2, -0.08465608465608465, m4); y[2] = Ops::fma3(k, x[5], y[2]); y[5] = Ops::fma3(k, x[2], y[5]); }
      { k = Ops::fmac(Lam[5], -0.08465608465608465, Ops::mulc(Lam[2], 0.40634920634920635)); y[2] = Ops::fma3(k, x[6], y[2]); y[6] = Ops::fma3(k, x[2], y[6]); }
      { k = Ops::fmac(Lam[5], 0.08465608465608465, Ops::fmac(Lam[2], -0.8507936507936508, m3)); y[2] = Ops::fma3(k, x[7], y[2]); y[7] = Ops::fma3(k, x[2], y[7]); }
      { k = Ops::fmac(Lam[5], 0.25396825396825395, Ops::fmac(Lam[2], 1.5576719576719578, m2)); y[2] = Ops::fma3(k, x[8], y[2]); y[8] = Ops::fma3(k, x[2], y[8]); }
      { k = Ops::fmac(Lam[5], -0.08465608465608465, Ops::mulc(Lam[4], 0.40634920634920635)); y[2] = Ops::fma3(k, x[9], y[2]); y[9] = Ops::fma3(k, x[2], y[9]); }
      { k = Ops::fmac(Lam[5], 0.08465608465608465, Ops::fmac(Lam[4], -0.8507936507936508, m3)); y[2] = Ops::fma3(k, x[10], y[2]); y[10] = Ops::fma3(k, x[2], y[10]); }
      { k = Ops::fmac(Lam[5], 0.25396825396825395, Ops::fmac(Lam[4], 1.5576719576719578, m2)); y[2] = Ops::fma3(k, x[11], y[2]); y[11] = Ops::fma3(k, x[2], y[11]); }
      { k = Ops::fmac(w34, -0.21164021164021163, m6); y[2] = Ops::fma3(k, x[12], y[2]); y[12] = Ops::fma3(k, x[2], y[12]); }
      { k = Ops::fmac(w34, -0.21164021164021163, m6); y[2] = Ops::fma3(k, x[13], y[2]); y[13] = Ops::fma3(k, x[2], y[13]); }
      { k = Ops::fmac(w2, 0.6349206349206349, Ops::fmac(Lam[5], 0.4656084656084656, m2)); y[2] = Ops::fma3(k, x[14], y[2]); y[14] = Ops::fma3(k, x[2], y[14]); }
      { k = Ops::fmac(w11, 4.1989417989417985, Ops::fmac(Lam[0], 3.657142857142857, m7)); y[3] = Ops::fma3(k, x[3], y[3]); }
      { k = Ops::fmac(Lam[3], -1.5238095238095237, Ops::fmac(Lam[1], 1.0497354497354496, Ops::fmac(Lam[0], -1.3206349206349206, m8))); y[3] = Ops::fma3(k, x[4], y[3]); y[4] = Ops::fma3(k, x[3], y[4]); }
      { k = Ops::fmac(w9, 0.6772486772486772, Ops::fmac(Lam[1], -0.6772486772486772, m9)); y[3] = Ops::fma3(k, x[5], y[3]); y[5] = Ops::fma3(k, x[3], y[5]); }
      { k = Ops::fmac(w31, 4.1989417989417985, Ops::fmac(Lam[0], 1.8285714285714285, m10)); y[3] = Ops::fma3(k, x[6], y[3]); y[6] = Ops::fma3(k, x[3], y[6]); }
      { k = Ops::fmac(w17, -0.728042328042328, Ops::fmac(Lam[2], -0.9312169312169312, Ops::fmac(Lam[1], -0.5925925925925926, m11))); y[3] = Ops::fma3(k, x[7], y[3]); y[7] = Ops::fma3(k, x[3], y[7]); }
      { k = Ops::fmac(w7, 0.20317460317460317, Ops::fmac(Lam[4], 0.6772486772486772, Ops::fmac(Lam[2], 0.4740740740740741, m12))); y[3] = Ops::fma3(k, x[8], y[3]); y[8] = Ops::fma3(k, x[3], y[8]); }
      { k = Ops::fmac(w4, 0.20317460317460317, Ops::fmac(Lam[2], 0.6772486772486772, Ops::fmac(Lam[1], 0.4740740740740741, m12))); y[3] = Ops::fma3(k, x[9], y[3]); y[9] = Ops::fma3(k, x[3], y[9]); }
      { k = Ops::fmac(w4, 0.08465608465608465, Ops::fmac(Lam[2], 0.3047619047619048, Ops::fmac(Lam[1], 0.2201058201058201, m13))); y[3] = Ops::fma3(k, x[10], y[3]); y[10] = Ops::fma3(k, x[3], y[10]); }
      { k = Ops::fmac(w5, 0.20317460317460317, Ops::fmac(Lam[2], 0.40634920634920635, m14)); y[3] = Ops::fma3(k, x[11], y[3]); y[11] = Ops::fma3(k, x[3], y[11]); }
      { k = Ops::fmac(w28, 5.147089947089947, Ops::fmac(Lam[0], 0.2708994708994709, m10)); y[3] = Ops::fma3(k, x[12], y[3]); y[12] = Ops::fma3(k, x[3], y[12]); }
      { k = Ops::fmac(w4, -0.5417989417989418, Ops::fmac(Lam[2], -0.8126984126984127, Ops::fmac(Lam[0], 0.8126984126984127, m14))); y[3] = Ops::fma3(k, x[13], y[3]); y[13] = Ops::fma3(k, x[3], y[13]); }
      { k = Ops::fmac(w29, -1.3544973544973544, Ops::fmac(Lam[0], 0.2708994708994709, m15)); y[3] = Ops::fma3(k, x[14], y[3]); y[14] = Ops::fma3(k, x[3], y[14]); }
      { k = Ops::fmac(w9, 4.901587301587302, Ops::fmac(Lam[1], 3.8857142857142857, m16)); y[4] = Ops::fma3(k, x[4], y[4]); }
      { k = Ops::fmac(Lam[3], -1.3206349206349206, Ops::fmac(Lam[1], 1.0497354497354496, Ops::fmac(Lam[0], -1.5238095238095237, m8))); y[4] = Ops::fma3(k, x[5], y[4]); y[5] = Ops::fma3(k, x[4], y[5]); }
      { k = Ops::fmac(w17, -0.728042328042328, Ops::fmac(Lam[2], -0.5925925925925926, Ops::fmac(Lam[1], -0.9312169312169312, m11))); y[4] = Ops::fma3(k, x[6], y[4]); y[6] = Ops::fma3(k, x[4], y[6]); }
      { k = Ops::fmac(w31, -0.7873015873015873, Ops::fmac(Lam[0], -0.2920634920634921, m17)); y[4] = Ops::fma3(k, x[7], y[4]); y[7] = Ops::fma3(k, x[4], y[7]); }
      { k = Ops::fmac(w7, 0.08465608465608465, Ops::fmac(Lam[4], 0.3047619047619048, Ops::fmac(Lam[2], 0.2201058201058201, m13))); y[4] = Ops::fma3(k, x[8], y[4]); y[8] = Ops::fma3(k, x[4], y[8]); }
      { k = Ops::fmac(w25, -1.5238095238095237, Ops::fmac(Lam[4], -0.5925925925925926, Ops::fmac(Lam[1], -0.9312169312169312, m11))); y[4] = Ops::fma3(k, x[9], y[4]); y[9] = Ops::fma3(k, x[4], y[9]); }
      { k = Ops::fmac(w27, -0.7873015873015873, Ops::fmac(Lam[3], -0.2920634920634921, m17)); y[4] = Ops::fma3(k, x[10], y[4]); y[10] = Ops::fma3(k, x[4], y[10]); }
      { k = Ops::fmac(w11, 0.08465608465608465, Ops::fmac(Lam[4], 0.2201058201058201, Ops::fmac(Lam[2], 0.3047619047619048, m13))); y[4] = Ops::fma3(k, x[11], y[4]); y[11] = Ops::fma3(k, x[4], y[11]); }
      { k = Ops::fmac(w35, 1.8285714285714285, Ops::fmac(Lam[3], -1.0158730158730158, m18)); y[4] = Ops::fma3(k, x[12], y[4]); y[12] = Ops::fma3(k, x[4], y[12]); }
      { k = Ops::fmac(w36, 1.8285714285714285, Ops::fmac(Lam[0], -1.0158730158730158, m18)); y[4] = Ops::fma3(k, x[13], y[4]); y[13] = Ops::fma3(k, x[4], y[13]); }
      { k = Ops::fmac(w9, -0.6095238095238096, Ops::fmac(w2, -1.4222222222222223, Ops::fmac(Lam[1], -1.0158730158730158, m19))); y[4] = Ops::fma3(k, x[14], y[4]); y[14] = Ops::fma3(k, x[4], y[14]); }
      { k = Ops::fmac(w7, 4.1989417989417985, Ops::fmac(Lam[3], 3.657142857142857, m7)); y[5] = Ops::fma3(k, x[5], y[5]); }
      { k = Ops::fmac(w8, 0.20317460317460317, Ops::fmac(Lam[4], 0.6772486772486772, Ops::fmac(Lam[1], 0.4740740740740741, m12))); y[5] = Ops::fma3(k, x[6], y[5]); y[6] = Ops::fma3(k, x[5], y[6]); }
      { k = Ops::fmac(w8, 0.08465608465608465, Ops::fmac(Lam[4], 0.3047619047619048, Ops::fmac(Lam[1], 0.2201058201058201, m13))); y[5] = Ops::fma3(k, x[7], y[5]); y[7] = Ops::fma3(k, x[5], y[7]); }
      { k = Ops::fmac(w3, 0.20317460317460317, Ops::fmac(Lam[4], 0.40634920634920635, m14)); y[5] = Ops::fma3(k, x[8], y[5]); y[8] = Ops::fma3(k, x[5], y[8]); }
      { k = Ops::fmac(w27, 4.1989417989417985, Ops::fmac(Lam[3], 1.8285714285714285, m10)); y[5] = Ops::fma3(k, x[9], y[5]); y[9] = Ops::fma3(k, x[5], y[9]); }
      { k = Ops::fmac(w25, -1.5238095238095237, Ops::fmac(Lam[4], -0.9312169312169312, Ops::fmac(Lam[1], -0.5925925925925926, m11))); y[5] = Ops::fma3(k, x[10], y[5]); y[10] = Ops::fma3(k, x[5], y[10]); }
      { k = Ops::fmac(w11, 0.20317460317460317, Ops::fmac(Lam[4], 0.4740740740740741, Ops::fmac(Lam[2], 0.6772486772486772, m12))); y[5] = Ops::fma3(k, x[11], y[5]); y[11] = Ops::fma3(k, x[5], y[11]); }
      { k = Ops::fmac(w8, -0.5417989417989418, Ops::fmac(Lam[4], -0.8126984126984127, Ops::fmac(Lam[3], 0.8126984126984127, m14))); y[5] = Ops::fma3(k, x[12], y[5]); y[12] = Ops::fma3(k, x[5], y[12]); }
      { k = Ops::fmac(w32, 5.147089947089947, Ops::fmac(Lam[3], 0.2708994708994709, m10)); y[5] = Ops::fma3(k, x[13], y[5]); y[13] = Ops::fma3(k, x[5], y[13]); }
      { k = Ops::fmac(w33, -1.3544973544973544, Ops::fmac(Lam[3], 0.2708994708994709, m15)); y[5] = Ops::fma3(k, x[14], y[5]); y[14] = Ops::fma3(k, x[5], y[14]); }
      { k = Ops::fmac(w12, 4.1989417989417985, Ops::fmac(Lam[0], 3.657142857142857, m7)); y[6] = Ops::fma3(k, x[6], y[6]); }
      { k = Ops::fmac(Lam[5], -1.5238095238095237, Ops::fmac(Lam[2], 1.0497354497354496, Ops::fmac(Lam[0], -1.3206349206349206, m8))); y[6] = Ops::fma3(k, x[7], y[6]); y[7] = Ops::fma3(k, x[6], y[7]); }
      { k = Ops::fmac(w10, 0.6772486772486772, Ops::fmac(Lam[2], -0.6772486772486772, m9)); y[6] = Ops::fma3(k, x[8], y[6]); y[8] = Ops::fma3(k, x[6], y[8]); }
      { k = Ops::fmac(w6, 0.20317460317460317, Ops::fmac(Lam[1], 0.40634920634920635, m14)); y[6] = Ops::fma3(k, x[9], y[6]); y[9] = Ops::fma3(k, x[6], y[9]); }
      { k = Ops::fmac(w14, 0.08465608465608465, Ops::fmac(Lam[2], 0.2201058201058201, Ops::fmac(Lam[1], 0.3047619047619048, m13))); y[6] = Ops::fma3(k, x[10], y[6]); y[10] = Ops::fma3(k, x[6], y[10]); }
      { k = Ops::fmac(w14, 0.20317460317460317, Ops::fmac(Lam[2], 0.4740740740740741, Ops::fmac(Lam[1], 0.6772486772486772, m12))); y[6] = Ops::fma3(k, x[11], y[6]); y[11] = Ops::fma3(k, x[6], y[11]); }
      { k = Ops::fmac(w23, 5.147089947089947, Ops::fmac(Lam[0], 0.2708994708994709, m10)); y[6] = Ops::fma3(k, x[12], y[6]); y[12] = Ops::fma3(k, x[6], y[12]); }
      { k = Ops::fmac(w24, -1.3544973544973544, Ops::fmac(Lam[0], 0.2708994708994709, m15)); y[6] = Ops::fma3(k, x[13], y[6]); y[13] = Ops::fma3(k, x[6], y[13]); }
      { k = Ops::fmac(w14, -0.5417989417989418, Ops::fmac(Lam[1], -0.8126984126984127, Ops::fmac(Lam[0], 0.8126984126984127, m14))); y[6] = Ops::fma3(k, x[14], y[6]); y[14] = Ops::fma3(k, x[6], y[14]); }
      { k = Ops::fmac(w10, 4.901587301587302, Ops::fmac(Lam[2], 3.8857142857142857, m16)); y[7] = Ops::fma3(k, x[7], y[7]); }
      { k = Ops::fmac(Lam[5], -1.3206349206349206, Ops::fmac(Lam[2], 1.0497354497354496, Ops::fmac(Lam[0], -1.5238095238095237, m8))); y[7] = Ops::fma3(k, x[8], y[7]); y[8] = Ops::fma3(k, x[7], y[8]); }
      { k = Ops::fmac(w12, 0.08465608465608465, Ops::fmac(Lam[4], 0.2201058201058201, Ops::fmac(Lam[1], 0.3047619047619048, m13))); y[7] = Ops::fma3(k, x[9], y[7]); y[9] = Ops::fma3(k, x[7], y[9]); }
      { k = Ops::fmac(w22, -0.7873015873015873, Ops::fmac(Lam[5], -0.2920634920634921, m17)); y[7] = Ops::fma3(k, x[10], y[7]); y[10] = Ops::fma3(k, x[7], y[10]); }
      { k = Ops::fmac(w20, -1.5238095238095237, Ops::fmac(Lam[4], -0.5925925925925926, Ops::fmac(Lam[2], -0.9312169312169312, m11))); y[7] = Ops::fma3(k, x[11], y[7]); y[11] = Ops::fma3(k, x[7], y[11]); }
      { k = Ops::fmac(w35, 1.8285714285714285, Ops::fmac(Lam[5], -1.0158730158730158, m18)); y[7] = Ops::fma3(k, x[12], y[7]); y[12] = Ops::fma3(k, x[7], y[12]); }
      { k = Ops::fmac(w10, -0.6095238095238096, Ops::fmac(w1, -1.4222222222222223, Ops::fmac(Lam[2], -1.0158730158730158, m19))); y[7] = Ops::fma3(k, x[13], y[7]); y[13] = Ops::fma3(k, x[7], y[13]); }
      { k = Ops::fmac(w37, 1.8285714285714285, Ops::fmac(Lam[0], -1.0158730158730158, m18)); y[7] = Ops::fma3(k, x[14], y[7]); y[14] = Ops::fma3(k, x[7], y[14]); }
      { k = Ops::fmac(w8, 4.1989417989417985, Ops::fmac(Lam[5], 3.657142857142857, m7)); y[8] = Ops::fma3(k, x[8], y[8]); }
      { k = Ops::fmac(w12, 0.20317460317460317, Ops::fmac(Lam[4], 0.4740740740740741, Ops::fmac(Lam[1], 0.6772486772486772, m12))); y[8] = Ops::fma3(k, x[9], y[8]); y[9] = Ops::fma3(k, x[8], y[9]); }
      { k = Ops::fmac(w20, -1.5238095238095237, Ops::fmac(Lam[4], -0.9312169312169312, Ops::fmac(Lam[2], -0.5925925925925926, m11))); y[8] = Ops::fma3(k, x[10], y[8]); y[10] = Ops::fma3(k, x[8], y[10]); }
      { k = Ops::fmac(w22, 4.1989417989417985, Ops::fmac(Lam[5], 1.8285714285714285, m10)); y[8] = Ops::fma3(k, x[11], y[8]); y[11] = Ops::fma3(k, x[8], y[11]); }
      { k = Ops::fmac(w7, -0.5417989417989418, Ops::fmac(Lam[5], 0.8126984126984127, Ops::fmac(Lam[4], -0.8126984126984127, m14))); y[8] = Ops::fma3(k, x[12], y[8]); y[12] = Ops::fma3(k, x[8], y[12]); }
      { k = Ops::fmac(w33, -1.3544973544973544, Ops::fmac(Lam[5], 0.2708994708994709, m15)); y[8] = Ops::fma3(k, x[13], y[8]); y[13] = Ops::fma3(k, x[8], y[13]); }
      { k = Ops::fmac(w32, 5.147089947089947, Ops::fmac(Lam[5], 0.2708994708994709, m10)); y[8] = Ops::fma3(k, x[14], y[8]); y[14] = Ops::fma3(k, x[8], y[14]); }
      { k = Ops::fmac(w14, 4.1989417989417985, Ops::fmac(Lam[3], 3.657142857142857, m7)); y[9] = Ops::fma3(k, x[9], y[9]); }
      { k = Ops::fmac(Lam[5], -1.5238095238095237, Ops::fmac(Lam[4], 1.0497354497354496, Ops::fmac(Lam[3], -1.3206349206349206, m8))); y[9] = Ops::fma3(k, x[10], y[9]); y[10] = Ops::fma3(k, x[9], y[10]); }
      { k = Ops::fmac(w13, 0.6772486772486772, Ops::fmac(Lam[4], -0.6772486772486772, m9)); y[9] = Ops::fma3(k, x[11], y[9]); y[11] = Ops::fma3(k, x[9], y[11]); }
      { k = Ops::fmac(w24, -1.3544973544973544, Ops::fmac(Lam[3], 0.2708994708994709, m15)); y[9] = Ops::fma3(k, x[12], y[9]); y[12] = Ops::fma3(k, x[9], y[12]); }
      { k = Ops::fmac(w23, 5.147089947089947, Ops::fmac(Lam[3], 0.2708994708994709, m10)); y[9] = Ops::fma3(k, x[13], y[9]); y[13] = Ops::fma3(k, x[9], y[13]); }
      { k = Ops::fmac(w12, -0.5417989417989418, Ops::fmac(Lam[3], 0.8126984126984127, Ops::fmac(Lam[1], -0.8126984126984127, m14))); y[9] = Ops::fma3(k, x[14], y[9]); y[14] = Ops::fma3(k, x[9], y[14]); }
      { k = Ops::fmac(w13, 4.901587301587302, Ops::fmac(Lam[4], 3.8857142857142857, m16)); y[10] = Ops::fma3(k, x[10], y[10]); }
      { k = Ops::fmac(Lam[5], -1.3206349206349206, Ops::fmac(Lam[4], 1.0497354497354496, Ops::fmac(Lam[3], -1.5238095238095237, m8))); y[10] = Ops::fma3(k, x[11], y[10]); y[11] = Ops::fma3(k, x[10], y[11]); }
      { k = Ops::fmac(w13, -0.6095238095238096, Ops::fmac(w0, -1.4222222222222223, Ops::fmac(Lam[4], -1.0158730158730158, m19))); y[10] = Ops::fma3(k, x[12], y[10]); y[12] = Ops::fma3(k, x[10], y[12]); }
      { k = Ops::fmac(w36, 1.8285714285714285, Ops::fmac(Lam[5], -1.0158730158730158, m18)); y[10] = Ops::fma3(k, x[13], y[10]); y[13] = Ops::fma3(k, x[10], y[13]); }
      { k = Ops::fmac(w37, 1.8285714285714285, Ops::fmac(Lam[3], -1.0158730158730158, m18)); y[10] = Ops::fma3(k, x[14], y[10]); y[14] = Ops::fma3(k, x[10], y[14]); }
      { k = Ops::fmac(w4, 4.1989417989417985, Ops::fmac(Lam[5], 3.657142857142857, m7)); y[11] = Ops::fma3(k, x[11], y[11]); }
      { k = Ops::fmac(w29, -1.3544973544973544, Ops::fmac(Lam[5], 0.2708994708994709, m15)); y[11] = Ops::fma3(k, x[12], y[11]); y[12] = Ops::fma3(k, x[11], y[12]); }
      { k = Ops::fmac(w11, -0.5417989417989418, Ops::fmac(Lam[5], 0.8126984126984127, Ops::fmac(Lam[2], -0.8126984126984127, m14))); y[11] = Ops::fma3(k, x[13], y[11]); y[13] = Ops::fma3(k, x[11], y[13]); }
      { k = Ops::fmac(w28, 5.147089947089947, Ops::fmac(Lam[5], 0.2708994708994709, m10)); y[11] = Ops::fma3(k, x[14], y[11]); y[14] = Ops::fma3(k, x[11], y[14]); }
      { k = Ops::fmac(w16, 11.377777777777778, m20); y[12] = Ops::fma3(k, x[12], y[12]); }
      { k = Ops::fmac(w9, -1.6253968253968254, Ops::fmac(w6, 1.6253968253968254, Ops::fmac(Lam[1], 4.876190476190477, m21))); y[12] = Ops::fma3(k, x[13], y[12]); y[13] = Ops::fma3(k, x[12], y[13]); }
      { k = Ops::fmac(w10, -1.6253968253968254, Ops::fmac(w5, 1.6253968253968254, Ops::fmac(Lam[2], 4.876190476190477, m21))); y[12] = Ops::fma3(k, x[14], y[12]); y[14] = Ops::fma3(k, x[12], y[14]); }
      { k = Ops::fmac(w16, 11.377777777777778, m20); y[13] = Ops::fma3(k, x[13], y[13]); }
      { k = Ops::fmac(w13, -1.6253968253968254, Ops::fmac(w3, 1.6253968253968254, Ops::fmac(Lam[4], 4.876190476190477, m21))); y[13] = Ops::fma3(k, x[14], y[13]); y[14] = Ops::fma3(k, x[13], y[14]); }
      { k = Ops::fmac(w16, 11.377777777777778, m20); y[14] = Ops::fma3(k, x[14], y[14]); }
    }
    else if constexpr (STIFF) {
      const typename Ops::T w0 = Ops::add(Lam[1], Lam[2]);
      const typename Ops::T w1 = Ops::add(Lam[1], Lam[4]);
      const typename Ops::T w2 = Ops::add(Lam[2], Lam[4]);
      const typename Ops::T w3 = Ops::add(Lam[0], w0);
      const typename Ops::T w4 = Ops::add(Lam[3], Lam[4]);
      const typename Ops::T w5 = Ops::add(Lam[3], w1);
      const typename Ops::T w6 = Ops::add(Lam[5], w2);
      const typename Ops::T w7 = Ops::add(Lam[0], Lam[1]);
      const typename Ops::T w8 = Ops::add(Lam[0], Lam[2]);
      const typename Ops::T w9 = Ops::add(Lam[0], Lam[3]);
      const typename Ops::T w10 = Ops::add(Lam[0], Lam[5]);
      const typename Ops::T w11 = Ops::add(Lam[1], Lam[3]);
      const typename Ops::T w12 = Ops::add(Lam[2], Lam[5]);
      const typename Ops::T w13 = Ops::add(Lam[3], Lam[5]);
      const typename Ops::T w14 = Ops::add(Lam[4], Lam[5]);
      const typename Ops::T w15 = Ops::add(Lam[5], w3);
      const typename Ops::T w16 = Ops::add(w4, w15);
      const typename Ops::T w17 = Ops::fmac(Lam[4], 2.0930232558139537, Lam[0]);
      const typename Ops::T w18 = Ops::fmac(Lam[4], 1.7692307692307692, Lam[0]);
      const typename Ops::T w19 = Ops::fmac(w0, 0.2, Lam[0]);
      const typename Ops::T w20 = Ops::fmac(Lam[5], 0.4777777777777778, Lam[1]);
      const typename Ops::T w21 = Ops::fmac(Lam[5], 0.5652173913043478, Lam[1]);
      const typename Ops::T w22 = Ops::fmac(w2, 0.5, Lam[1]);
      const typename Ops::T w23 = Ops::fmac(w6, 0.631578947368421, Lam[1]);
      const typename Ops::T w24 = Ops::fmac(w6, 0.4, Lam[1]);
      const typename Ops::T w25 = Ops::fmac(Lam[3], 0.4777777777777778, Lam[2]);
      const typename Ops::T w26 = Ops::fmac(Lam[3], 0.5652173913043478, Lam[2]);
      const typename Ops::T w27 = Ops::fmac(w1, 0.5, Lam[2]);
      const typename Ops::T w28 = Ops::fmac(w5, 0.631578947368421, Lam[2]);
      const typename Ops::T w29 = Ops::fmac(w5, 0.4, Lam[2]);
      const typename Ops::T w30 = Ops::fmac(w1, 0.2, Lam[3]);
      const typename Ops::T w31 = Ops::fmac(w0, 0.5, Lam[4]);
      const typename Ops::T w32 = Ops::fmac(w3, 0.631578947368421, Lam[4]);
      const typename Ops::T w33 = Ops::fmac(w3, 0.4, Lam[4]);
      const typename Ops::T w34 = Ops::fmac(w2, 0.2, Lam[5]);
      const typename Ops::T w35 = Ops::fmac(w18, 1.4444444444444444, w0);
      const typename Ops::T w36 = Ops::fmac(w26, 2.5555555555555554, w1);
      const typename Ops::T w37 = Ops::fmac(w21, 2.5555555555555554, w2);
      { k = Ops::mulc(Lam[0], 0.746031746031746); y[0] = Ops::mul(k, x[0]); }
      { k = Ops::mulc(Lam[1], -0.11322751322751323); y[0] = Ops::fma3(k, x[1], y[0]); y[1] = Ops::mul(k, x[0]); }
      { k = Ops::mulc(Lam[2], -0.11322751322751323); y[0] = Ops::fma3(k, x[2], y[0]); y[2] = Ops::mul(k, x[0]); }
      { k = Ops::fmac(Lam[1], 1.5576719576719578, Ops::mulc(Lam[0], 0.25396825396825395)); y[0] = Ops::fma3(k, x[3], y[0]); y[3] = Ops::mul(k, x[0]); }
      { k = Ops::fmac(Lam[1], -0.8507936507936508, Ops::mulc(Lam[0], 0.08465608465608465)); y[0] = Ops::fma3(k, x[4], y[0]); y[4] = Ops::mul(k, x[0]); }
      { k = Ops::fmac(Lam[1], 0.40634920634920635, Ops::mulc(Lam[0], -0.08465608465608465)); y[0] = Ops::fma3(k, x[5], y[0]); y[5] = Ops::mul(k, x[0]); }
      { k = Ops::fmac(Lam[2], 1.5576719576719578, Ops::mulc(Lam[0], 0.25396825396825395)); y[0] = Ops::fma3(k, x[6], y[0]); y[6] = Ops::mul(k, x[0]); }
      { k = Ops::fmac(Lam[2], -0.8507936507936508, Ops::mulc(Lam[0], 0.08465608465608465)); y[0] = Ops::fma3(k, x[7], y[0]); y[7] = Ops::mul(k, x[0]); }
      { k = Ops::fmac(Lam[2], 0.40634920634920635, Ops::mulc(Lam[0], -0.08465608465608465)); y[0] = Ops::fma3(k, x[8], y[0]); y[8] = Ops::mul(k, x[0]); }
      { k = Ops::mulc(w0, -0.08465608465608465); y[0] = Ops::fma3(k, x[9], y[0]); y[9] = Ops::mul(k, x[0]); }
      { k = Ops::mulc(w0, -0.08465608465608465); y[0] = Ops::fma3(k, x[10], y[0]); y[10] = Ops::mul(k, x[0]); }
      { k = Ops::mulc(w0, -0.08465608465608465); y[0] = Ops::fma3(k, x[11], y[0]); y[11] = Ops::mul(k, x[0]); }
      { k = Ops::fmac(w0, 0.6349206349206349, Ops::mulc(Lam[0], 0.4656084656084656)); y[0] = Ops::fma3(k, x[12], y[0]); y[12] = Ops::mul(k, x[0]); }
      { k = Ops::mulc(w19, -0.21164021164021163); y[0] = Ops::fma3(k, x[13], y[0]); y[13] = Ops::mul(k, x[0]); }
      { k = Ops::mulc(w19, -0.21164021164021163); y[0] = Ops::fma3(k, x[14], y[0]); y[14] = Ops::mul(k, x[0]); }
      { k = Ops::mulc(Lam[3], 0.746031746031746); y[1] = Ops::fma3(k, x[1], y[1]); }
      { k = Ops::mulc(Lam[4], -0.11322751322751323); y[1] = Ops::fma3(k, x[2], y[1]); y[2] = Ops::fma3(k, x[1], y[2]); }
      { k = Ops::fmac(Lam[3], -0.08465608465608465, Ops::mulc(Lam[1], 0.40634920634920635)); y[1] = Ops::fma3(k, x[3], y[1]); y[3] = Ops::fma3(k, x[1], y[3]); }
      { k = Ops::fmac(Lam[3], 0.08465608465608465, Ops::mulc(Lam[1], -0.8507936507936508)); y[1] = Ops::fma3(k, x[4], y[1]); y[4] = Ops::fma3(k, x[1], y[4]); }
      { k = Ops::fmac(Lam[3], 0.25396825396825395, Ops::mulc(Lam[1], 1.5576719576719578)); y[1] = Ops::fma3(k, x[5], y[1]); y[5] = Ops::fma3(k, x[1], y[5]); }
      { k = Ops::mulc(w1, -0.08465608465608465); y[1] = Ops::fma3(k, x[6], y[1]); y[6] = Ops::fma3(k, x[1], y[6]); }
      { k = Ops::mulc(w1, -0.08465608465608465); y[1] = Ops::fma3(k, x[7], y[1]); y[7] = Ops::fma3(k, x[1], y[7]); }
      { k = Ops::mulc(w1, -0.08465608465608465); y[1] = Ops::fma3(k, x[8], y[1]); y[8] = Ops::fma3(k, x[1], y[8]); }
      { k = Ops::fmac(Lam[4], 1.5576719576719578, Ops::mulc(Lam[3], 0.25396825396825395)); y[1] = Ops::fma3(k, x[9], y[1]); y[9] = Ops::fma3(k, x[1], y[9]); }
      { k = Ops::fmac(Lam[4], -0.8507936507936508, Ops::mulc(Lam[3], 0.08465608465608465)); y[1] = Ops::fma3(k, x[10], y[1]); y[10] = Ops::fma3(k, x[1], y[10]); }
      { k = Ops::fmac(Lam[4], 0.40634920634920635, Ops::mulc(Lam[3], -0.08465608465608465)); y[1] = Ops::fma3(k, x[11], y[1]); y[11] = Ops::fma3(k, x[1], y[11]); }
      { k = Ops::mulc(w30, -0.21164021164021163); y[1] = Ops::fma3(k, x[12], y[1]); y[12] = Ops::fma3(k, x[1], y[12]); }
      { k = Ops::fmac(w1, 0.6349206349206349, Ops::mulc(Lam[3], 0.4656084656084656)); y[1] = Ops::fma3(k, x[13], y[1]); y[13] = Ops::fma3(k, x[1], y[13]); }
      { k = Ops::mulc(w30, -0.21164021164021163); y[1] = Ops::fma3(k, x[14], y[1]); y[14] = Ops::fma3(k, x[1], y[14]); }
      { k = Ops::mulc(Lam[5], 0.746031746031746); y[2] = Ops::fma3(k, x[2], y[2]); }
      { k = Ops::mulc(w2, -0.08465608465608465); y[2] = Ops::fma3(k, x[3], y[2]); y[3] = Ops::fma3(k, x[2], y[3]); }
      { k = Ops::mulc(w2, -0.08465608465608465); y[2] = Ops::fma3(k, x[4], y[2]); y[4] = Ops::fma3(k, x[2], y[4]); }
      { k = Ops::mulc(w2, -0.08465608465608465); y[2] = Ops::fma3(k, x[5], y[2]); y[5] = Ops::fma3(k, x[2], y[5]); }
      { k = Ops::fmac(Lam[5], -0.08465608465608465, Ops::mulc(Lam[2], 0.40634920634920635)); y[2] = Ops::fma3(k, x[6], y[2]); y[6] = Ops::fma3(k, x[2], y[6]); }
      { k = Ops::fmac(Lam[5], 0.08465608465608465, Ops::mulc(Lam[2], -0.8507936507936508)); y[2] = Ops::fma3(k, x[7], y[2]); y[7] = Ops::fma3(k, x[2], y[7]); }
      { k = Ops::fmac(Lam[5], 0.25396825396825395, Ops::mulc(Lam[2], 1.5576719576719578)); y[2] = Ops::fma3(k, x[8], y[2]); y[8] = Ops::fma3(k, x[2], y[8]); }
      { k = Ops::fmac(Lam[5], -0.08465608465608465, Ops::mulc(Lam[4], 0.40634920634920635)); y[2] = Ops::fma3(k, x[9], y[2]); y[9] = Ops::fma3(k, x[2], y[9]); }
      { k = Ops::fmac(Lam[5], 0.08465608465608465, Ops::mulc(Lam[4], -0.8507936507936508)); y[2] = Ops::fma3(k, x[10], y[2]); y[10] = Ops::fma3(k, x[2], y[10]); }
      { k = Ops::fmac(Lam[5], 0.25396825396825395, Ops::mulc(Lam[4], 1.5576719576719578)); y[2] = Ops::fma3(k, x[11], y[2]); y[11] = Ops::fma3(k, x[2], y[11]); }
      { k = Ops::mulc(w34, -0.21164021164021163); y[2] = Ops::fma3(k, x[12], y[2]); y[12] = Ops::fma3(k, x[2], y[12]); }
      { k = Ops::mulc(w34, -0.21164021164021163); y[2] = Ops::fma3(k, x[13], y[2]); y[13] = Ops::fma3(k, x[2], y[13]); }
      { k = Ops::fmac(w2, 0.6349206349206349, Ops::mulc(Lam[5], 0.4656084656084656)); y[2] = Ops::fma3(k, x[14], y[2]); y[14] = Ops::fma3(k, x[2], y[14]); }
      { k = Ops::fmac(w11, 4.1989417989417985, Ops::mulc(Lam[0], 3.657142857142857)); y[3] = Ops::fma3(k, x[3], y[3]); }
      { k = Ops::fmac(Lam[3], -1.5238095238095237, Ops::fmac(Lam[1], 1.0497354497354496, Ops::mulc(Lam[0], -1.3206349206349206))); y[3] = Ops::fma3(k, x[4], y[3]); y[4] = Ops::fma3(k, x[3], y[4]); }
      { k = Ops::fmac(w9, 0.6772486772486772, Ops::mulc(Lam[1], -0.6772486772486772)); y[3] = Ops::fma3(k, x[5], y[3]); y[5] = Ops::fma3(k, x[3], y[5]); }
      { k = Ops::fmac(w31, 4.1989417989417985, Ops::mulc(Lam[0], 1.8285714285714285)); y[3] = Ops::fma3(k, x[6], y[3]); y[6] = Ops::fma3(k, x[3], y[6]); }
      { k = Ops::fmac(w17, -0.728042328042328, Ops::fmac(Lam[2], -0.9312169312169312, Ops::mulc(Lam[1], -0.5925925925925926))); y[3] = Ops::fma3(k, x[7], y[3]); y[7] = Ops::fma3(k, x[3], y[7]); }
      { k = Ops::fmac(w7, 0.20317460317460317, Ops::fmac(Lam[4], 0.6772486772486772, Ops::mulc(Lam[2], 0.4740740740740741))); y[3] = Ops::fma3(k, x[8], y[3]); y[8] = Ops::fma3(k, x[3], y[8]); }
      { k = Ops::fmac(w4, 0.20317460317460317, Ops::fmac(Lam[2], 0.6772486772486772, Ops::mulc(Lam[1], 0.4740740740740741))); y[3] = Ops::fma3(k, x[9], y[3]); y[9] = Ops::fma3(k, x[3], y[9]); }
      { k = Ops::fmac(w4, 0.08465608465608465, Ops::fmac(Lam[2], 0.3047619047619048, Ops::mulc(Lam[1], 0.2201058201058201))); y[3] = Ops::fma3(k, x[10], y[3]); y[10] = Ops::fma3(k, x[3], y[10]); }
      { k = Ops::fmac(w5, 0.20317460317460317, Ops::mulc(Lam[2], 0.40634920634920635)); y[3] = Ops::fma3(k, x[11], y[3]); y[11] = Ops::fma3(k, x[3], y[11]); }
      { k = Ops::fmac(w28, 5.147089947089947, Ops::mulc(Lam[0], 0.2708994708994709)); y[3] = Ops::fma3(k, x[12], y[3]); y[12] = Ops::fma3(k, x[3], y[12]); }
      { k = Ops::fmac(w4, -0.5417989417989418, Ops::fmac(Lam[2], -0.8126984126984127, Ops::mulc(Lam[0], 0.8126984126984127))); y[3] = Ops::fma3(k, x[13], y[3]); y[13] = Ops::fma3(k, x[3], y[13]); }
      { k = Ops::fmac(w29, -1.3544973544973544, Ops::mulc(Lam[0], 0.2708994708994709)); y[3] = Ops::fma3(k, x[14], y[3]); y[14] = Ops::fma3(k, x[3], y[14]); }
      { k = Ops::fmac(w9, 4.901587301587302, Ops::mulc(Lam[1], 3.8857142857142857)); y[4] = Ops::fma3(k, x[4], y[4]); }
      { k = Ops::fmac(Lam[3], -1.3206349206349206, Ops::fmac(Lam[1], 1.0497354497354496, Ops::mulc(Lam[0], -1.5238095238095237))); y[4] = Ops::fma3(k, x[5], y[4]); y[5] = Ops::fma3(k, x[4], y[5]); }
      { k = Ops::fmac(w17, -0.728042328042328, Ops::fmac(Lam[2], -0.5925925925925926, Ops::mulc(Lam[1], -0.9312169312169312))); y[4] = Ops::fma3(k, x[6], y[4]); y[6] = Ops::fma3(k, x[4], y[6]); }
      { k = Ops::fmac(w31, -0.7873015873015873, Ops::mulc(Lam[0], -0.2920634920634921)); y[4] = Ops::fma3(k, x[7], y[4]); y[7] = Ops::fma3(k, x[4], y[7]); }
      { k = Ops::fmac(w7, 0.08465608465608465, Ops::fmac(Lam[4], 0.3047619047619048, Ops::mulc(Lam[2], 0.2201058201058201))); y[4] = Ops::fma3(k, x[8], y[4]); y[8] = Ops::fma3(k, x[4], y[8]); }
      { k = Ops::fmac(w25, -1.5238095238095237, Ops::fmac(Lam[4], -0.5925925925925926, Ops::mulc(Lam[1], -0.9312169312169312))); y[4] = Ops::fma3(k, x[9], y[4]); y[9] = Ops::fma3(k, x[4], y[9]); }
      { k = Ops::fmac(w27, -0.7873015873015873, Ops::mulc(Lam[3], -0.2920634920634921)); y[4] = Ops::fma3(k, x[10], y[4]); y[10] = Ops::fma3(k, x[4], y[10]); }
      { k = Ops::fmac(w11, 0.08465608465608465, Ops::fmac(Lam[4], 0.2201058201058201, Ops::mulc(Lam[2], 0.3047619047619048))); y[4] = Ops::fma3(k, x[11], y[4]); y[11] = Ops::fma3(k, x[4], y[11]); }
      { k = Ops::fmac(w35, 1.8285714285714285, Ops::mulc(Lam[3], -1.0158730158730158)); y[4] = Ops::fma3(k, x[12], y[4]); y[12] = Ops::fma3(k, x[4], y[12]); }
      { k = Ops::fmac(w36, 1.8285714285714285, Ops::mulc(Lam[0], -1.0158730158730158)); y[4] = Ops::fma3(k, x[13], y[4]); y[13] = Ops::fma3(k, x[4], y[13]); }
      { k = Ops::fmac(w9, -0.6095238095238096, Ops::fmac(w2, -1.4222222222222223, Ops::mulc(Lam[1], -1.0158730158730158))); y[4] = Ops::fma3(k, x[14], y[4]); y[14] = Ops::fma3(k, x[4], y[14]); }
      { k = Ops::fmac(w7, 4.1989417989417985, Ops::mulc(Lam[3], 3.657142857142857)); y[5] = Ops::fma3(k, x[5], y[5]); }
      { k = Ops::fmac(w8, 0.20317460317460317, Ops::fmac(Lam[4], 0.6772486772486772, Ops::mulc(Lam[1], 0.4740740740740741))); y[5] = Ops::fma3(k, x[6], y[5]); y[6] = Ops::fma3(k, x[5], y[6]); }
      { k = Ops::fmac(w8, 0.08465608465608465, Ops::fmac(Lam[4], 0.3047619047619048, Ops::mulc(Lam[1], 0.2201058201058201))); y[5] = Ops::fma3(k, x[7], y[5]); y[7] = Ops::fma3(k, x[5], y[7]); }
      { k = Ops::fmac(w3, 0.20317460317460317, Ops::mulc(Lam[4], 0.40634920634920635)); y[5] = Ops::fma3(k, x[8], y[5]); y[8] = Ops::fma3(k, x[5], y[8]); }
      { k = Ops::fmac(w27, 4.1989417989417985, Ops::mulc(Lam[3], 1.8285714285714285)); y[5] = Ops::fma3(k, x[9], y[5]); y[9] = Ops::fma3(k, x[5], y[9]); }
      { k = Ops::fmac(w25, -1.5238095238095237, Ops::fmac(Lam[4], -0.9312169312169312, Ops::mulc(Lam[1], -0.5925925925925926))); y[5] = Ops::fma3(k, x[10], y[5]); y[10] = Ops::fma3(k, x[5], y[10]); }
      { k = Ops::fmac(w11, 0.20317460317460317, Ops::fmac(Lam[4], 0.4740740740740741, Ops::mulc(Lam[2], 0.6772486772486772))); y[5] = Ops::fma3(k, x[11], y[5]); y[11] = Ops::fma3(k, x[5], y[11]); }
      { k = Ops::fmac(w8, -0.5417989417989418, Ops::fmac(Lam[4], -0.8126984126984127, Ops::mulc(Lam[3], 0.8126984126984127))); y[5] = Ops::fma3(k, x[12], y[5]); y[12] = Ops::fma3(k, x[5], y[12]); }
      { k = Ops::fmac(w32, 5.147089947089947, Ops::mulc(Lam[3], 0.2708994708994709)); y[5] = Ops::fma3(k, x[13], y[5]); y[13] = Ops::fma3(k, x[5], y[13]); }
      { k = Ops::fmac(w33, -1.3544973544973544, Ops::mulc(Lam[3], 0.2708994708994709)); y[5] = Ops::fma3(k, x[14], y[5]); y[14] = Ops::fma3(k, x[5], y[14]); }
      { k = Ops::fmac(w12, 4.1989417989417985, Ops::mulc(Lam[0], 3.657142857142857)); y[6] = Ops::fma3(k, x[6], y[6]); }
      { k = Ops::fmac(Lam[5], -1.5238095238095237, Ops::fmac(Lam[2], 1.0497354497354496, Ops::mulc(Lam[0], -1.3206349206349206))); y[6] = Ops::fma3(k, x[7], y[6]); y[7] = Ops::fma3(k, x[6], y[7]); }
      { k = Ops::fmac(w10, 0.6772486772486772, Ops::mulc(Lam[2], -0.6772486772486772)); y[6] = Ops::fma3(k, x[8], y[6]); y[8] = Ops::fma3(k, x[6], y[8]); }
      { k = Ops::fmac(w6, 0.20317460317460317, Ops::mulc(Lam[1], 0.40634920634920635)); y[6] = Ops::fma3(k, x[9], y[6]); y[9] = Ops::fma3(k, x[6], y[9]); }
      { k = Ops::fmac(w14, 0.08465608465608465, Ops::fmac(Lam[2], 0.2201058201058201, Ops::mulc(Lam[1], 0.3047619047619048))); y[6] = Ops::fma3(k, x[10], y[6]); y[10] = Ops::fma3(k, x[6], y[10]); }
      { k = Ops::fmac(w14, 0.20317460317460317, Ops::fmac(Lam[2], 0.4740740740740741, Ops::mulc(Lam[1], 0.6772486772486772))); y[6] = Ops::fma3(k, x[11], y[6]); y[11] = Ops::fma3(k, x[6], y[11]); }
      { k = Ops::fmac(w23, 5.147089947089947, Ops::mulc(Lam[0], 0.2708994708994709)); y[6] = Ops::fma3(k, x[12], y[6]); y[12] = Ops::fma3(k, x[6], y[12]); }
      { k = Ops::fmac(w24, -1.3544973544973544, Ops::mulc(Lam[0], 0.2708994708994709)); y[6] = Ops::fma3(k, x[13], y[6]); y[13] = Ops::fma3(k, x[6], y[13]); }
      { k = Ops::fmac(w14, -0.5417989417989418, Ops::fmac(Lam[1], -0.8126984126984127, Ops::mulc(Lam[0], 0.8126984126984127))); y[6] = Ops::fma3(k, x[14], y[6]); y[14] = Ops::fma3(k, x[6], y[14]); }
      { k = Ops::fmac(w10, 4.901587301587302, Ops::mulc(Lam[2], 3.8857142857142857)); y[7] = Ops::fma3(k, x[7], y[7]); }
      { k = Ops::fmac(Lam[5], -1.3206349206349206, Ops::fmac(Lam[2], 1.0497354497354496, Ops::mulc(Lam[0], -1.5238095238095237))); y[7] = Ops::fma3(k, x[8], y[7]); y[8] = Ops::fma3(k, x[7], y[8]); }
      { k = Ops::fmac(w12, 0.08465608465608465, Ops::fmac(Lam[4], 0.2201058201058201, Ops::mulc(Lam[1], 0.3047619047619048))); y[7] = Ops::fma3(k, x[9], y[7]); y[9] = Ops::fma3(k, x[7], y[9]); }
      { k = Ops::fmac(w22, -0.7873015873015873, Ops::mulc(Lam[5], -0.2920634920634921)); y[7] = Ops::fma3(k, x[10], y[7]); y[10] = Ops::fma3(k, x[7], y[10]); }
      { k = Ops::fmac(w20, -1.5238095238095237, Ops::fmac(Lam[4], -0.5925925925925926, Ops::mulc(Lam[2], -0.9312169312169312))); y[7] = Ops::fma3(k, x[11], y[7]); y[11] = Ops::fma3(k, x[7], y[11]); }
      { k = Ops::fmac(w35, 1.8285714285714285, Ops::mulc(Lam[5], -1.0158730158730158)); y[7] = Ops::fma3(k, x[12], y[7]); y[12] = Ops::fma3(k, x[7], y[12]); }
      { k = Ops::fmac(w10, -0.6095238095238096, Ops::fmac(w1, -1.4222222222222223, Ops::mulc(Lam[2], -1.0158730158730158))); y[7] = Ops::fma3(k, x[13], y[7]); y[13] = Ops::fma3(k, x[7], y[13]); }
      { k = Ops::fmac(w37, 1.8285714285714285, Ops::mulc(Lam[0], -1.0158730158730158)); y[7] = Ops::fma3(k, x[14], y[7]); y[14] = Ops::fma3(k, x[7], y[14]); }
      { k = Ops::fmac(w8, 4.1989417989417985, Ops::mulc(Lam[5], 3.657142857142857)); y[8] = Ops::fma3(k, x[8], y[8]); }
      { k = Ops::fmac(w12, 0.20317460317460317, Ops::fmac(Lam[4], 0.4740740740740741, Ops::mulc(Lam[1], 0.6772486772486772))); y[8] = Ops::fma3(k, x[9], y[8]); y[9] = Ops::fma3(k, x[8], y[9]); }
      { k = Ops::fmac(w20, -1.5238095238095237, Ops::fmac(Lam[4], -0.9312169312169312, Ops::mulc(Lam[2], -0.5925925925925926))); y[8] = Ops::fma3(k, x[10], y[8]); y[10] = Ops::fma3(k, x[8], y[10]); }
      { k = Ops::fmac(w22, 4.1989417989417985, Ops::mulc(Lam[5], 1.8285714285714285)); y[8] = Ops::fma3(k, x[11], y[8]); y[11] = Ops::fma3(k, x[8], y[11]); }
      { k = Ops::fmac(w7, -0.5417989417989418, Ops::fmac(Lam[5], 0.8126984126984127, Ops::mulc(Lam[4], -0.8126984126984127))); y[8] = Ops::fma3(k, x[12], y[8]); y[12] = Ops::fma3(k, x[8], y[12]); }
      { k = Ops::fmac(w33, -1.3544973544973544, Ops::mulc(Lam[5], 0.2708994708994709)); y[8] = Ops::fma3(k, x[13], y[8]); y[13] = Ops::fma3(k, x[8], y[13]); }
      { k = Ops::fmac(w32, 5.147089947089947, Ops::mulc(Lam[5], 0.2708994708994709)); y[8] = Ops::fma3(k, x[14], y[8]); y[14] = Ops::fma3(k, x[8], y[14]); }
      { k = Ops::fmac(w14, 4.1989417989417985, Ops::mulc(Lam[3], 3.657142857142857)); y[9] = Ops::fma3(k, x[9], y[9]); }
      { k = Ops::fmac(Lam[5], -1.5238095238095237, Ops::fmac(Lam[4], 1.0497354497354496, Ops::mulc(Lam[3], -1.3206349206349206))); y[9] = Ops::fma3(k, x[10], y[9]); y[10] = Ops::fma3(k, x[9], y[10]); }
      { k = Ops::fmac(w13, 0.6772486772486772, Ops::mulc(Lam[4], -0.6772486772486772)); y[9] = Ops::fma3(k, x[11], y[9]); y[11] = Ops::fma3(k, x[9], y[11]); }
      { k = Ops::fmac(w24, -1.3544973544973544, Ops::mulc(Lam[3], 0.2708994708994709)); y[9] = Ops::fma3(k, x[12], y[9]); y[12] = Ops::fma3(k, x[9], y[12]); }
      { k = Ops::fmac(w23, 5.147089947089947, Ops::mulc(Lam[3], 0.2708994708994709)); y[9] = Ops::fma3(k, x[13], y[9]); y[13] = Ops::fma3(k, x[9], y[13]); }
      { k = Ops::fmac(w12, -0.5417989417989418, Ops::fmac(Lam[3], 0.8126984126984127, Ops::mulc(Lam[1], -0.8126984126984127))); y[9] = Ops::fma3(k, x[14], y[9]); y[14] = Ops::fma3(k, x[9], y[14]); }
      { k = Ops::fmac(w13, 4.901587301587302, Ops::mulc(Lam[4], 3.8857142857142857)); y[10] = Ops::fma3(k, x[10], y[10]); }
      { k = Ops::fmac(Lam[5], -1.3206349206349206, Ops::fmac(Lam[4], 1.0497354497354496, Ops::mulc(Lam[3], -1.5238095238095237))); y[10] = Ops::fma3(k, x[11], y[10]); y[11] = Ops::fma3(k, x[10], y[11]); }
      { k = Ops::fmac(w13, -0.6095238095238096, Ops::fmac(w0, -1.4222222222222223, Ops::mulc(Lam[4], -1.0158730158730158))); y[10] = Ops::fma3(k, x[12], y[10]); y[12] = Ops::fma3(k, x[10], y[12]); }
      { k = Ops::fmac(w36, 1.8285714285714285, Ops::mulc(Lam[5], -1.0158730158730158)); y[10] = Ops::fma3(k, x[13], y[10]); y[13] = Ops::fma3(k, x[10], y[13]); }
      { k = Ops::fmac(w37, 1.8285714285714285, Ops::mulc(Lam[3], -1.0158730158730158)); y[10] = Ops::fma3(k, x[14], y[10]); y[14] = Ops::fma3(k, x[10], y[14]); }
      { k = Ops::fmac(w4, 4.1989417989417985, Ops::mulc(Lam[5], 3.657142857142857)); y[11] = Ops::fma3(k, x[11], y[11]); }
      { k = Ops::fmac(w29, -1.3544973544973544, Ops::mulc(Lam[5], 0.2708994708994709)); y[11] = Ops::fma3(k, x[12], y[11]); y[12] = Ops::fma3(k, x[11], y[12]); }
      { k = Ops::fmac(w11, -0.5417989417989418, Ops::fmac(Lam[5], 0.8126984126984127, Ops::mulc(Lam[2], -0.8126984126984127))); y[11] = Ops::fma3(k, x[13], y[11]); y[13] = Ops::fma3(k, x[11], y[13]); }
      { k = Ops::fmac(w28, 5.147089947089947, Ops::mulc(Lam[5], 0.2708994708994709)); y[11] = Ops::fma3(k, x[14], y[11]); y[14] = Ops::fma3(k, x[11], y[14]); }
      { k = Ops::mulc(w16, 11.377777777777778); y[12] = Ops::fma3(k, x[12], y[12]); }
      { k = Ops::fmac(w9, -1.6253968253968254, Ops::fmac(w6, 1.6253968253968254, Ops::mulc(Lam[1], 4.876190476190477))); y[12] = Ops::fma3(k, x[13], y[12]); y[13] = Ops::fma3(k, x[12], y[13]); }
      { k = Ops::fmac(w10, -1.6253968253968254, Ops::fmac(w5, 1.6253968253968254, Ops::mulc(Lam[2], 4.876190476190477))); y[12] = Ops::fma3(k, x[14], y[12]); y[14] = Ops::fma3(k, x[12], y[14]); }
      { k = Ops::mulc(w16, 11.377777777777778); y[13] = Ops::fma3(k, x[13], y[13]); }
      { k = Ops::fmac(w13, -1.6253968253968254, Ops::fmac(w3, 1.6253968253968254, Ops::mulc(Lam[4], 4.876190476190477))); y[13] = Ops::fma3(k, x[14], y[13]); y[14] = Ops::fma3(k, x[13], y[14]); }
      { k = Ops::mulc(w16, 11.377777777777778); y[14] = Ops::fma3(k, x[14], y[14]); }
    }
    else if constexpr (MASS) {
      const typename Ops::T m0 = Ops::mulc(vol, 0.0051146384479717815);
      const typename Ops::T m1 = Ops::mulc(vol, -0.0004761904761904762);
      const typename Ops::T m2 = Ops::mulc(vol, 0.0028218694885361554);
      const typename Ops::T m3 = Ops::mulc(vol, -0.0014109347442680777);
      const typename Ops::T m4 = Ops::mulc(vol, -0.0019753086419753087);
      const typename Ops::T m5 = Ops::mulc(vol, -0.00021164021164021165);
      const typename Ops::T m6 = Ops::mulc(vol, -0.0028218694885361554);
      const typename Ops::T m7 = Ops::mulc(vol, 0.045149911816578486);
      const typename Ops::T m8 = Ops::mulc(vol, -0.022574955908289243);
      const typename Ops::T m9 = Ops::mulc(vol, 0.013544973544973546);
      const typename Ops::T m10 = Ops::mulc(vol, 0.022574955908289243);
      const typename Ops::T m11 = Ops::mulc(vol, -0.016931216931216932);
      const typename Ops::T m12 = Ops::mulc(vol, 0.009029982363315696);
      const typename Ops::T m13 = Ops::mulc(vol, 0.001128747795414462);
      const typename Ops::T m14 = Ops::mulc(vol, 0.004514991181657848);
      const typename Ops::T m15 = Ops::mulc(vol, -0.004514991181657848);
      const typename Ops::T m16 = Ops::mulc(vol, 0.05587301587301587);
      const typename Ops::T m17 = Ops::mulc(vol, 0.0008465608465608466);
      const typename Ops::T m18 = Ops::mulc(vol, 0.006772486772486773);
      const typename Ops::T m19 = Ops::mulc(vol, -0.013544973544973546);
      const typename Ops::T m20 = Ops::mulc(vol, 0.18962962962962962);
      const typename Ops::T m21 = Ops::mulc(vol, -0.02708994708994709);
      { k = m0; y[0] = Ops::mul(k, x[0]); }
      { k = m1; y[0] = Ops::fma3(k, x[1], y[0]); y[1] = Ops::mul(k, x[0]); }
      { k = m1; y[0] = Ops::fma3(k, x[2], y[0]); y[2] = Ops::mul(k, x[0]); }
      { k = m2; y[0] = Ops::fma3(k, x[3], y[0]); y[3] = Ops::mul(k, x[0]); }
      { k = m3; y[0] = Ops::fma3(k, x[4], y[0]); y[4] = Ops::mul(k, x[0]); }
      { k = m2; y[0] = Ops::fma3(k, x[6], y[0]); y[6] = Ops::mul(k, x[0]); }
      { k = m3; y[0] = Ops::fma3(k, x[7], y[0]); y[7] = Ops::mul(k, x[0]); }
      { k = m4; y[0] = Ops::fma3(k, x[9], y[0]); y[9] = Ops::mul(k, x[0]); }
      { k = m5; y[0] = Ops::fma3(k, x[10], y[0]); y[10] = Ops::mul(k, x[0]); }
      { k = m4; y[0] = Ops::fma3(k, x[11], y[0]); y[11] = Ops::mul(k, x[0]); }
      { k = m2; y[0] = Ops::fma3(k, x[12], y[0]); y[12] = Ops::mul(k, x[0]); }
      { k = m6; y[0] = Ops::fma3(k, x[13], y[0]); y[13] = Ops::mul(k, x[0]); }
      { k = m6; y[0] = Ops::fma3(k, x[14], y[0]); y[14] = Ops::mul(k, x[0]); }
      { k = m0; y[1] = Ops::fma3(k, x[1], y[1]); }
      { k = m1; y[1] = Ops::fma3(k, x[2], y[1]); y[2] = Ops::fma3(k, x[1], y[2]); }
      { k = m3; y[1] = Ops::fma3(k, x[4], y[1]); y[4] = Ops::fma3(k, x[1], y[4]); }
      { k = m2; y[1] = Ops::fma3(k, x[5], y[1]); y[5] = Ops::mul(k, x[1]); }
      { k = m4; y[1] = Ops::fma3(k, x[6], y[1]); y[6] = Ops::fma3(k, x[1], y[6]); }
      { k = m5; y[1] = Ops::fma3(k, x[7], y[1]); y[7] = Ops::fma3(k, x[1], y[7]); }
      { k = m4; y[1] = Ops::fma3(k, x[8], y[1]); y[8] = Ops::mul(k, x[1]); }
      { k = m2; y[1] = Ops::fma3(k, x[9], y[1]); y[9] = Ops::fma3(k, x[1], y[9]); }
      { k = m3; y[1] = Ops::fma3(k, x[10], y[1]); y[10] = Ops::fma3(k, x[1], y[10]); }
      { k = m6; y[1] = Ops::fma3(k, x[12], y[1]); y[12] = Ops::fma3(k, x[1], y[12]); }
      { k = m2; y[1] = Ops::fma3(k, x[13], y[1]); y[13] = Ops::fma3(k, x[1], y[13]); }
      { k = m6; y[1] = Ops::fma3(k, x[14], y[1]); y[14] = Ops::fma3(k, x[1], y[14]); }
      { k = m0; y[2] = Ops::fma3(k, x[2], y[2]); }
      { k = m4; y[2] = Ops::fma3(k, x[3], y[2]); y[3] = Ops::fma3(k, x[2], y[3]); }
      { k = m5; y[2] = Ops::fma3(k, x[4], y[2]); y[4] = Ops::fma3(k, x[2], y[4]); }
      { k = m4; y[2] = Ops::fma3(k, x[5], y[2]); y[5] = Ops::fma3(k, x[2], y[5]); }
      { k = m3; y[2] = Ops::fma3(k, x[7], y[2]); y[7] = Ops::fma3(k, x[2], y[7]); }
      { k = m2; y[2] = Ops::fma3(k, x[8], y[2]); y[8] = Ops::fma3(k, x[2], y[8]); }
      { k = m3; y[2] = Ops::fma3(k, x[10], y[2]); y[10] = Ops::fma3(k, x[2], y[10]); }
      { k = m2; y[2] = Ops::fma3(k, x[11], y[2]); y[11] = Ops::fma3(k, x[2], y[11]); }
      { k = m6; y[2] = Ops::fma3(k, x[12], y[2]); y[12] = Ops::fma3(k, x[2], y[12]); }
      { k = m6; y[2] = Ops::fma3(k, x[13], y[2]); y[13] = Ops::fma3(k, x[2], y[13]); }
      { k = m2; y[2] = Ops::fma3(k, x[14], y[2]); y[14] = Ops::fma3(k, x[2], y[14]); }
      { k = m7; y[3] = Ops::fma3(k, x[3], y[3]); }
      { k = m8; y[3] = Ops::fma3(k, x[4], y[3]); y[4] = Ops::fma3(k, x[3], y[4]); }
      { k = m9; y[3] = Ops::fma3(k, x[5], y[3]); y[5] = Ops::fma3(k, x[3], y[5]); }
      { k = m10; y[3] = Ops::fma3(k, x[6], y[3]); y[6] = Ops::fma3(k, x[3], y[6]); }
      { k = m11; y[3] = Ops::fma3(k, x[7], y[3]); y[7] = Ops::fma3(k, x[3], y[7]); }
      { k = m12; y[3] = Ops::fma3(k, x[8], y[3]); y[8] = Ops::fma3(k, x[3], y[8]); }
      { k = m12; y[3] = Ops::fma3(k, x[9], y[3]); y[9] = Ops::fma3(k, x[3], y[9]); }
      { k = m13; y[3] = Ops::fma3(k, x[10], y[3]); y[10] = Ops::fma3(k, x[3], y[10]); }
      { k = m14; y[3] = Ops::fma3(k, x[11], y[3]); y[11] = Ops::fma3(k, x[3], y[11]); }
      { k = m10; y[3] = Ops::fma3(k, x[12], y[3]); y[12] = Ops::fma3(k, x[3], y[12]); }
      { k = m14; y[3] = Ops::fma3(k, x[13], y[3]); y[13] = Ops::fma3(k, x[3], y[13]); }
      { k = m15; y[3] = Ops::fma3(k, x[14], y[3]); y[14] = Ops::fma3(k, x[3], y[14]); }
      { k = m16; y[4] = Ops::fma3(k, x[4], y[4]); }
      { k = m8; y[4] = Ops::fma3(k, x[5], y[4]); y[5] = Ops::fma3(k, x[4], y[5]); }
      { k = m11; y[4] = Ops::fma3(k, x[6], y[4]); y[6] = Ops::fma3(k, x[4], y[6]); }
      { k = m17; y[4] = Ops::fma3(k, x[7], y[4]); y[7] = Ops::fma3(k, x[4], y[7]); }
      { k = m13; y[4] = Ops::fma3(k, x[8], y[4]); y[8] = Ops::fma3(k, x[4], y[8]); }
      { k = m11; y[4] = Ops::fma3(k, x[9], y[4]); y[9] = Ops::fma3(k, x[4], y[9]); }
      { k = m17; y[4] = Ops::fma3(k, x[10], y[4]); y[10] = Ops::fma3(k, x[4], y[10]); }
      { k = m13; y[4] = Ops::fma3(k, x[11], y[4]); y[11] = Ops::fma3(k, x[4], y[11]); }
      { k = m18; y[4] = Ops::fma3(k, x[12], y[4]); y[12] = Ops::fma3(k, x[4], y[12]); }
      { k = m18; y[4] = Ops::fma3(k, x[13], y[4]); y[13] = Ops::fma3(k, x[4], y[13]); }
      { k = m19; y[4] = Ops::fma3(k, x[14], y[4]); y[14] = Ops::fma3(k, x[4], y[14]); }
      { k = m7; y[5] = Ops::fma3(k, x[5], y[5]); }
      { k = m12; y[5] = Ops::fma3(k, x[6], y[5]); y[6] = Ops::fma3(k, x[5], y[6]); }
      { k = m13; y[5] = Ops::fma3(k, x[7], y[5]); y[7] = Ops::fma3(k, x[5], y[7]); }
      { k = m14; y[5] = Ops::fma3(k, x[8], y[5]); y[8] = Ops::fma3(k, x[5], y[8]); }
      { k = m10; y[5] = Ops::fma3(k, x[9], y[5]); y[9] = Ops::fma3(k, x[5], y[9]); }
      { k = m11; y[5] = Ops::fma3(k, x[10], y[5]); y[10] = Ops::fma3(k, x[5], y[10]); }
      { k = m12; y[5] = Ops::fma3(k, x[11], y[5]); y[11] = Ops::fma3(k, x[5], y[11]); }
      { k = m14; y[5] = Ops::fma3(k, x[12], y[5]); y[12] = Ops::fma3(k, x[5], y[12]); }
      { k = m10; y[5] = Ops::fma3(k, x[13], y[5]); y[13] = Ops::fma3(k, x[5], y[13]); }
      { k = m15; y[5] = Ops::fma3(k, x[14], y[5]); y[14] = Ops::fma3(k, x[5], y[14]); }
      { k = m7; y[6] = Ops::fma3(k, x[6], y[6]); }
      { k = m8; y[6] = Ops::fma3(k, x[7], y[6]); y[7] = Ops::fma3(k, x[6], y[7]); }
      { k = m9; y[6] = Ops::fma3(k, x[8], y[6]); y[8] = Ops::fma3(k, x[6], y[8]); }
      { k = m14; y[6] = Ops::fma3(k, x[9], y[6]); y[9] = Ops::fma3(k, x[6], y[9]); }
      { k = m13; y[6] = Ops::fma3(k, x[10], y[6]); y[10] = Ops::fma3(k, x[6], y[10]); }
      { k = m12; y[6] = Ops::fma3(k, x[11], y[6]); y[11] = Ops::fma3(k, x[6], y[11]); }
      { k = m10; y[6] = Ops::fma3(k, x[12], y[6]); y[12] = Ops::fma3(k, x[6], y[12]); }
      { k = m15; y[6] = Ops::fma3(k, x[13], y[6]); y[13] = Ops::fma3(k, x[6], y[13]); }
      { k = m14; y[6] = Ops::fma3(k, x[14], y[6]); y[14] = Ops::fma3(k, x[6], y[14]); }
      { k = m16; y[7] = Ops::fma3(k, x[7], y[7]); }
      { k = m8; y[7] = Ops::fma3(k, x[8], y[7]); y[8] = Ops::fma3(k, x[7], y[8]); }
      { k = m13; y[7] = Ops::fma3(k, x[9], y[7]); y[9] = Ops::fma3(k, x[7], y[9]); }
      { k = m17; y[7] = Ops::fma3(k, x[10], y[7]); y[10] = Ops::fma3(k, x[7], y[10]); }
      { k = m11; y[7] = Ops::fma3(k, x[11], y[7]); y[11] = Ops::fma3(k, x[7], y[11]); }
      { k = m18; y[7] = Ops::fma3(k, x[12], y[7]); y[12] = Ops::fma3(k, x[7], y[12]); }
      { k = m19; y[7] = Ops::fma3(k, x[13], y[7]); y[13] = Ops::fma3(k, x[7], y[13]); }
      { k = m18; y[7] = Ops::fma3(k, x[14], y[7]); y[14] = Ops::fma3(k, x[7], y[14]); }
      { k = m7; y[8] = Ops::fma3(k, x[8], y[8]); }
      { k = m12; y[8] = Ops::fma3(k, x[9], y[8]); y[9] = Ops::fma3(k, x[8], y[9]); }
      { k = m11; y[8] = Ops::fma3(k, x[10], y[8]); y[10] = Ops::fma3(k, x[8], y[10]); }
      { k = m10; y[8] = Ops::fma3(k, x[11], y[8]); y[11] = Ops::fma3(k, x[8], y[11]); }
      { k = m14; y[8] = Ops::fma3(k, x[12], y[8]); y[12] = Ops::fma3(k, x[8], y[12]); }
      { k = m15; y[8] = Ops::fma3(k, x[13], y[8]); y[13] = Ops::fma3(k, x[8], y[13]); }
      { k = m10; y[8] = Ops::fma3(k, x[14], y[8]); y[14] = Ops::fma3(k, x[8], y[14]); }
      { k = m7; y[9] = Ops::fma3(k, x[9], y[9]); }
      { k = m8; y[9] = Ops::fma3(k, x[10], y[9]); y[10] = Ops::fma3(k, x[9], y[10]); }
      { k = m9; y[9] = Ops::fma3(k, x[11], y[9]); y[11] = Ops::fma3(k, x[9], y[11]); }
      { k = m15; y[9] = Ops::fma3(k, x[12], y[9]); y[12] = Ops::fma3(k, x[9], y[12]); }
      { k = m10; y[9] = Ops::fma3(k, x[13], y[9]); y[13] = Ops::fma3(k, x[9], y[13]); }
      { k = m14; y[9] = Ops::fma3(k, x[14], y[9]); y[14] = Ops::fma3(k, x[9], y[14]); }
      { k = m16; y[10] = Ops::fma3(k, x[10], y[10]); }
      { k = m8; y[10] = Ops::fma3(k, x[11], y[10]); y[11] = Ops::fma3(k, x[10], y[11]); }
      { k = m19; y[10] = Ops::fma3(k, x[12], y[10]); y[12] = Ops::fma3(k, x[10], y[12]); }
      { k = m18; y[10] = Ops::fma3(k, x[13], y[10]); y[13] = Ops::fma3(k, x[10], y[13]); }
      { k = m18; y[10] = Ops::fma3(k, x[14], y[10]); y[14] = Ops::fma3(k, x[10], y[14]); }
      { k = m7; y[11] = Ops::fma3(k, x[11], y[11]); }
      { k = m15; y[11] = Ops::fma3(k, x[12], y[11]); y[12] = Ops::fma3(k, x[11], y[12]); }
      { k = m14; y[11] = Ops::fma3(k, x[13], y[11]); y[13] = Ops::fma3(k, x[11], y[13]); }
      { k = m10; y[11] = Ops::fma3(k, x[14], y[11]); y[14] = Ops::fma3(k, x[11], y[14]); }
      { k = m20; y[12] = Ops::fma3(k, x[12], y[12]); }
      { k = m21; y[12] = Ops::fma3(k, x[13], y[12]); y[13] = Ops::fma3(k, x[12], y[13]); }
      { k = m21; y[12] = Ops::fma3(k, x[14], y[12]); y[14] = Ops::fma3(k, x[12], y[14]); }
      { k = m20; y[13] = Ops::fma3(k, x[13], y[13]); }
      { k = m21; y[13] = Ops::fma3(k, x[14], y[13]); y[14] = Ops::fma3(k, x[13], y[14]); }
      { k = m20; y[14] = Ops::fma3(k, x[14], y[14]); }
    }
  }
  __host__ __device__ static constexpr int upper_index(int i, int j) {
    return i <= j ? i * 15 - (i * (i - 1)) / 2 + (j - i) : j * 15 - (j * (j - 1)) / 2 + (i - j);
  }
};

// ---- P1 Lagrange on the tetrahedron (4 nodes) ----
template <> struct Elem<3, 1> {
  static constexpr int ND = 4;
  static constexpr int NUP = 10;
  static constexpr int NLAM = 10;
  static constexpr int STIFF_TERMS = 10;
  // K[u] for u over the upper triangle (i <= j), row-major; Lam[k] over pairs (m <= n)
  static constexpr int STIFF_OPS = 10;  // after rewriting
  template <class Ops> __device__ __forceinline__ static void stiffness_upper(const typename Ops::T* Lam, typename Ops::T* K) {
    K[0] = Lam[0];
    K[1] = Lam[1];
    K[2] = Lam[2];
    K[3] = Lam[3];
    K[4] = Lam[4];
    K[5] = Lam[5];
    K[6] = Lam[6];
    K[7] = Lam[7];
    K[8] = Lam[8];
    K[9] = Lam[9];
  }
  template <class Ops> __device__ __forceinline__ static void helmholtz_upper(const typename Ops::T* Lam, const typename Ops::T& vol, typename Ops::T* K) {
    const typename Ops::T m0 = Ops::mulc(vol, 0.1);
    const typename Ops::T m1 = Ops::mulc(vol, 0.05);
    K[0] = Ops::fmac(Lam[0], 1.0, m0);
    K[1] = Ops::fmac(Lam[1], 1.0, m1);
    K[2] = Ops::fmac(Lam[2], 1.0, m1);
    K[3] = Ops::fmac(Lam[3], 1.0, m1);
    K[4] = Ops::fmac(Lam[4], 1.0, m0);
    K[5] = Ops::fmac(Lam[5], 1.0, m1);
    K[6] = Ops::fmac(Lam[6], 1.0, m1);
    K[7] = Ops::fmac(Lam[7], 1.0, m0);
    K[8] = Ops::fmac(Lam[8], 1.0, m1);
    K[9] = Ops::fmac(Lam[9], 1.0, m0);
  }
  template <class Ops> __device__ __forceinline__ static void mass_upper(const typename Ops::T& vol, typename Ops::T* K) {
    const typename Ops::T m0 = Ops::mulc(vol, 0.1);
    const typename Ops::T m1 = Ops::mulc(vol, 0.05);
    K[0] = m0;
    K[1] = m1;
    K[2] = m1;
    K[3] = m1;
    K[4] = m0;
    K[5] = m1;
    K[6] = m1;
    K[7] = m0;
    K[8] = m1;
    K[9] = m0;
  }
  template <class Ops, bool STIFF, bool MASS> __device__ __forceinline__ static void action_upper(const typename Ops::T* Lam, const typename Ops::T& vol, const typename Ops::T* x, typename Ops::T* y) {
    typename Ops::T k;
    if constexpr (STIFF && MASS) {
      const typename Ops::T m0 = Ops::mulc(vol, 0.1);
      const typename Ops::T m1 = Ops::mulc(vol, 0.05);
      { k = Ops::fmac(Lam[0], 1.0, m0); y[0] = Ops::mul(k, x[0]); }
      { k = Ops::fmac(Lam[1], 1.0, m1); y[0] = Ops::fma3(k, x[1], y[0]); y[1] = Ops::mul(k, x[0]); }
      { k = Ops::fmac(Lam[2], 1.0, m1); y[0] = Ops::fma3(k, x[2], y[0]); y[2] = Ops::mul(k, x[0]); }
      { k = Ops::fmac(Lam[3], 1.0, m1); y[0] = Ops::fma3(k, x[3], y[0]); y[3] = Ops::mul(k, x[0]); }
      { k = Ops::fmac(Lam[4], 1.0, m0); y[1] = Ops::fma3(k, x[1], y[1]); }
      { k = Ops::fmac(Lam[5], 1.0, m1); y[1] = Ops::fma3(k, x[2], y[1]); y[2] = Ops::fma3(k, x[1], y[2]); }
      { k = Ops::fmac(Lam[6], 1.0, m1); y[1] = Ops::fma3(k, x[3], y[1]); y[3] = Ops::fma3(k, x[1], y[3]); }
      { k = Ops::fmac(Lam[7], 1.0, m0); y[2] = Ops::fma3(k, x[2], y[2]); }
      { k = Ops::fmac(Lam[8], 1.0, m1); y[2] = Ops::fma3(k, x[3], y[2]); y[3] = Ops::fma3(k, x[2], y[3]); }
      { k = Ops::fmac(Lam[9], 1.0, m0); y[3] = Ops::fma3(k, x[3], y[3]); }
    }
    else if constexpr (STIFF) {
      { k = Lam[0]; y[0] = Ops::mul(k, x[0]); }
      { k = Lam[1]; y[0] = Ops::fma3(k, x[1], y[0]); y[1] = Ops::mul(k, x[0]); }
      { k = Lam[2]; y[0] = Ops::fma3(k, x[2], y[0]); y[2] = Ops::mul(k, x[0]); }
      { k = Lam[3]; y[0] = Ops::fma3(k, x[3], y[0]); y[3] = Ops::mul(k, x[0]); }
      { k = Lam[4]; y[1] = Ops::fma3(k, x[1], y[1]); }
      { k = Lam[5]; y[1] = Ops::fma3(k, x[2], y[1]); y[2] = Ops::fma3(k, x[1], y[2]); }
      { k = Lam[6]; y[1] = Ops::fma3(k, x[3], y[1]); y[3] = Ops::fma3(k, x[1], y[3]); }
      { k = Lam[7]; y[2] = Ops::fma3(k, x[2], y[2]); }
      { k = Lam[8]; y[2] = Ops::fma3(k, x[3], y[2]); y[3] = Ops::fma3(k, x[2], y[3]); }
      { k = Lam[9]; y[3] = Ops::fma3(k, x[3], y[3]); }
    }
    else if constexpr (MASS) {
      const typename Ops::T m0 = Ops::mulc(vol, 0.1);
      const typename Ops::T m1 = Ops::mulc(vol, 0.05);
      { k = m0; y[0] = Ops::mul(k, x[0]); }
      { k = m1; y[0] = Ops::fma3(k, x[1], y[0]); y[1] = Ops::mul(k, x[0]); }
      { k = m1; y[0] = Ops::fma3(k, x[2], y[0]); y[2] = Ops::mul(k, x[0]); }
      { k = m1; y[0] = Ops::fma3(k, x[3], y[0]); y[3] = Ops::mul(k, x[0]); }
      { k = m0; y[1] = Ops::fma3(k, x[1], y[1]); }
      { k = m1; y[1] = Ops::fma3(k, x[2], y[1]); y[2] = Ops::fma3(k, x[1], y[2]); }
      { k = m1; y[1] = Ops::fma3(k, x[3], y[1]); y[3] = Ops::fma3(k, x[1], y[3]); }
      { k = m0; y[2] = Ops::fma3(k, x[2], y[2]); }
      { k = m1; y[2] = Ops::fma3(k, x[3], y[2]); y[3] = Ops::fma3(k, x[2], y[3]); }
      { k = m0; y[3] = Ops::fma3(k, x[3], y[3]); }
    }
  }
  __host__ __device__ static constexpr int upper_index(int i, int j) {
    return i <= j ? i * 4 - (i * (i - 1)) / 2 + (j - i) : j * 4 - (j * (j - 1)) / 2 + (i - j);
  }
};

// ---- P2 Lagrange on the tetrahedron (10 nodes) ----
template <> struct Elem<3, 2> {
  static constexpr int ND = 10;
  static constexpr int NUP = 55;
  static constexpr int NLAM = 10;
  static constexpr int STIFF_TERMS = 136;
  // K[u] for u over the upper triangle (i <= j), row-major; Lam[k] over pairs (m <= n)
  static constexpr int STIFF_OPS = 118;  // after rewriting
  template <class Ops> __device__ __forceinline__ static void stiffness_upper(const typename Ops::T* Lam, typename Ops::T* K) {
    const typename Ops::T w0 = Ops::add(Lam[0], Lam[1]);
    const typename Ops::T w1 = Ops::add(Lam[1], Lam[5]);
    const typename Ops::T w2 = Ops::add(Lam[1], Lam[6]);
    const typename Ops::T w3 = Ops::add(Lam[2], Lam[3]);
    const typename Ops::T w4 = Ops::add(Lam[2], Lam[7]);
    const typename Ops::T w5 = Ops::add(Lam[3], Lam[8]);
    const typename Ops::T w6 = Ops::add(Lam[5], Lam[6]);
    const typename Ops::T w7 = Ops::add(Lam[6], Lam[9]);
    const typename Ops::T w8 = Ops::add(Lam[2], Lam[8]);
    const typename Ops::T w9 = Ops::add(Lam[5], Lam[7]);
    K[0] = Ops::mulc(Lam[0], 0.6);
    K[1] = Ops::mulc(Lam[1], -0.2);
    K[2] = Ops::mulc(Lam[2], -0.2);
    K[3] = Ops::mulc(Lam[3], -0.2);
    K[4] = Ops::fmac(Lam[1], 0.6, Ops::mulc(Lam[0], -0.2));
    K[5] = Ops::fmac(Lam[2], 0.6, Ops::mulc(Lam[0], -0.2));
    K[6] = Ops::fmac(Lam[3], 0.6, Ops::mulc(Lam[0], -0.2));
    K[7] = Ops::fmac(Lam[2], -0.2, Ops::mulc(Lam[1], -0.2));
    K[8] = Ops::fmac(Lam[3], -0.2, Ops::mulc(Lam[1], -0.2));
    K[9] = Ops::mulc(w3, -0.2);
    K[10] = Ops::mulc(Lam[4], 0.6);
    K[11] = Ops::mulc(Lam[5], -0.2);
    K[12] = Ops::mulc(Lam[6], -0.2);
    K[13] = Ops::fmac(Lam[4], -0.2, Ops::mulc(Lam[1], 0.6));
    K[14] = Ops::mulc(w1, -0.2);
    K[15] = Ops::mulc(w2, -0.2);
    K[16] = Ops::fmac(Lam[5], 0.6, Ops::mulc(Lam[4], -0.2));
    K[17] = Ops::fmac(Lam[6], 0.6, Ops::mulc(Lam[4], -0.2));
    K[18] = Ops::mulc(w6, -0.2);
    K[19] = Ops::mulc(Lam[7], 0.6);
    K[20] = Ops::mulc(Lam[8], -0.2);
    K[21] = Ops::fmac(Lam[5], -0.2, Ops::mulc(Lam[2], -0.2));
    K[22] = Ops::fmac(Lam[7], -0.2, Ops::mulc(Lam[2], 0.6));
    K[23] = Ops::mulc(w8, -0.2);
    K[24] = Ops::fmac(Lam[7], -0.2, Ops::mulc(Lam[5], 0.6));
    K[25] = Ops::fmac(Lam[8], -0.2, Ops::mulc(Lam[5], -0.2));
    K[26] = Ops::fmac(Lam[8], 0.6, Ops::mulc(Lam[7], -0.2));
    K[27] = Ops::mulc(Lam[9], 0.6);
    K[28] = Ops::fmac(Lam[6], -0.2, Ops::mulc(Lam[3], -0.2));
    K[29] = Ops::mulc(w5, -0.2);
    K[30] = Ops::fmac(Lam[9], -0.2, Ops::mulc(Lam[3], 0.6));
    K[31] = Ops::fmac(Lam[8], -0.2, Ops::mulc(Lam[6], -0.2));
    K[32] = Ops::fmac(Lam[9], -0.2, Ops::mulc(Lam[6], 0.6));
    K[33] = Ops::fmac(Lam[9], -0.2, Ops::mulc(Lam[8], 0.6));
    K[34] = Ops::fmac(w0, 1.6, Ops::mulc(Lam[4], 1.6));
    K[35] = Ops::fmac(w0, 0.8, Ops::fmac(Lam[5], 1.6, Ops::mulc(Lam[2], 0.8)));
    K[36] = Ops::fmac(w0, 0.8, Ops::fmac(Lam[6], 1.6, Ops::mulc(Lam[3], 0.8)));
    K[37] = Ops::fmac(w1, 0.8, Ops::fmac(Lam[4], 0.8, Ops::mulc(Lam[2], 1.6)));
    K[38] = Ops::fmac(w2, 0.8, Ops::fmac(Lam[4], 0.8, Ops::mulc(Lam[3], 1.6)));
    K[39] = Ops::fmac(w6, 0.8, Ops::mulc(w3, 0.8));
    K[40] = Ops::fmac(w4, 1.6, Ops::mulc(Lam[0], 1.6));
    K[41] = Ops::fmac(w3, 0.8, Ops::fmac(Lam[8], 1.6, Ops::mulc(Lam[0], 0.8)));
    K[42] = Ops::fmac(w4, 0.8, Ops::fmac(Lam[5], 0.8, Ops::mulc(Lam[1], 1.6)));
    K[43] = Ops::fmac(w5, 0.8, Ops::mulc(w1, 0.8));
    K[44] = Ops::fmac(w4, 0.8, Ops::fmac(Lam[8], 0.8, Ops::mulc(Lam[3], 1.6)));
    K[45] = Ops::fmac(Lam[9], 1.6, Ops::fmac(Lam[3], 1.6, Ops::mulc(Lam[0], 1.6)));
    K[46] = Ops::fmac(w8, 0.8, Ops::mulc(w2, 0.8));
    K[47] = Ops::fmac(w7, 0.8, Ops::fmac(Lam[3], 0.8, Ops::mulc(Lam[1], 1.6)));
    K[48] = Ops::fmac(w5, 0.8, Ops::fmac(Lam[9], 0.8, Ops::mulc(Lam[2], 1.6)));
    K[49] = Ops::fmac(w9, 1.6, Ops::mulc(Lam[4], 1.6));
    K[50] = Ops::fmac(w6, 0.8, Ops::fmac(Lam[8], 1.6, Ops::mulc(Lam[4], 0.8)));
    K[51] = Ops::fmac(w9, 0.8, Ops::fmac(Lam[8], 0.8, Ops::mulc(Lam[6], 1.6)));
    K[52] = Ops::fmac(w7, 1.6, Ops::mulc(Lam[4], 1.6));
    K[53] = Ops::fmac(w7, 0.8, Ops::fmac(Lam[8], 0.8, Ops::mulc(Lam[5], 1.6)));
    K[54] = Ops::fmac(Lam[9], 1.6, Ops::fmac(Lam[8], 1.6, Ops::mulc(Lam[7], 1.6)));
  }
  template <class Ops> __device__ __forceinline__ static void helmholtz_upper(const typename Ops::T* Lam, const typename Ops::T& vol, typename Ops::T* K) {
    const typename Ops::T w0 = Ops::add(Lam[0], Lam[1]);
    const typename Ops::T w1 = Ops::add(Lam[1], Lam[5]);
    const typename Ops::T w2 = Ops::add(Lam[1], Lam[6]);
    const typename Ops::T w3 = Ops::add(Lam[2], Lam[3]);
    const typename Ops::T w4 = Ops::add(Lam[2], Lam[7]);
    const typename Ops::T w5 = Ops::add(Lam[3], Lam[8]);
    const typename Ops::T w6 = Ops::add(Lam[5], Lam[6]);
    const typename Ops::T w7 = Ops::add(Lam[6], Lam[9]);
    const typename Ops::T w8 = Ops::add(Lam[2], Lam[8]);
    const typename Ops::T w9 = Ops::add(Lam[5], Lam[7]);
    const typename Ops::T m0 = Ops::mulc(vol, 0.014285714285714285);
    const typename Ops::T m1 = Ops::mulc(vol, 0.002380952380952381);
    const typename Ops::T m2 = Ops::mulc(vol, -0.009523809523809525);
    const typename Ops::T m3 = Ops::mulc(vol, -0.014285714285714285);
    const typename Ops::T m4 = Ops::mulc(vol, 0.0761904761904762);
    const typename Ops::T m5 = Ops::mulc(vol, 0.0380952380952381);
    const typename Ops::T m6 = Ops::mulc(vol, 0.01904761904761905);
    K[0] = Ops::fmac(Lam[0], 0.6, m0);
    K[1] = Ops::fmac(Lam[1], -0.2, m1);
    K[2] = Ops::fmac(Lam[2], -0.2, m1);
    K[3] = Ops::fmac(Lam[3], -0.2, m1);
    K[4] = Ops::fmac(Lam[1], 0.6, Ops::fmac(Lam[0], -0.2, m2));
    K[5] = Ops::fmac(Lam[2], 0.6, Ops::fmac(Lam[0], -0.2, m2));
    K[6] = Ops::fmac(Lam[3], 0.6, Ops::fmac(Lam[0], -0.2, m2));
    K[7] = Ops::fmac(Lam[2], -0.2, Ops::fmac(Lam[1], -0.2, m3));
    K[8] = Ops::fmac(Lam[3], -0.2, Ops::fmac(Lam[1], -0.2, m3));
    K[9] = Ops::fmac(w3, -0.2, m3);
    K[10] = Ops::fmac(Lam[4], 0.6, m0);
    K[11] = Ops::fmac(Lam[5], -0.2, m1);
    K[12] = Ops::fmac(Lam[6], -0.2, m1);
    K[13] = Ops::fmac(Lam[4], -0.2, Ops::fmac(Lam[1], 0.6, m2));
    K[14] = Ops::fmac(w1, -0.2, m3);
    K[15] = Ops::fmac(w2, -0.2, m3);
    K[16] = Ops::fmac(Lam[5], 0.6, Ops::fmac(Lam[4], -0.2, m2));
    K[17] = Ops::fmac(Lam[6], 0.6, Ops::fmac(Lam[4], -0.2, m2));
    K[18] = Ops::fmac(w6, -0.2, m3);
    K[19] = Ops::fmac(Lam[7], 0.6, m0);
    K[20] = Ops::fmac(Lam[8], -0.2, m1);
    K[21] = Ops::fmac(Lam[5], -0.2, Ops::fmac(Lam[2], -0.2, m3));
    K[22] = Ops::fmac(Lam[7], -0.2, Ops::fmac(Lam[2], 0.6, m2));
    K[23] = Ops::fmac(w8, -0.2, m3);
    K[24] = Ops::fmac(Lam[7], -0.2, Ops::fmac(Lam[5], 0.6, m2));
    K[25] = Ops::fmac(Lam[8], -0.2, Ops::fmac(Lam[5], -0.2, m3));
    K[26] = Ops::fmac(Lam[8], 0.6, Ops::fmac(Lam[7], -0.2, m2));
    K[27] = Ops::fmac(Lam[9], 0.6, m0);
    K[28] = Ops::fmac(Lam[6], -0.2, Ops::fmac(Lam[3], -0.2, m3));
    K[29] = Ops::fmac(w5, -0.2, m3);
    K[30] = Ops::fmac(Lam[9], -0.2, Ops::fmac(Lam[3], 0.6, m2));
    K[31] = Ops::fmac(Lam[8], -0.2, Ops::fmac(Lam[6], -0.2, m3));
    K[32] = Ops::fmac(Lam[9], -0.2, Ops::fmac(Lam[6], 0.6, m2));
    K[33] = Ops::fmac(Lam[9], -0.2, Ops::fmac(Lam[8], 0.6, m2));
    K[34] = Ops::fmac(w0, 1.6, Ops::fmac(Lam[4], 1.6, m4));
    K[35] = Ops::fmac(w0, 0.8, Ops::fmac(Lam[5], 1.6, Ops::fmac(Lam[2], 0.8, m5)));
    K[36] = Ops::fmac(w0, 0.8, Ops::fmac(Lam[6], 1.6, Ops::fmac(Lam[3], 0.8, m5)));
    K[37] = Ops::fmac(w1, 0.8, Ops::fmac(Lam[4], 0.8, Ops::fmac(Lam[2], 1.6, m5)));
    K[38] = Ops::fmac(w2, 0.8, Ops::fmac(Lam[4], 0.8, Ops::fmac(Lam[3], 1.6, m5)));
    K[39] = Ops::fmac(w6, 0.8, Ops::fmac(w3, 0.8, m6));
    K[40] = Ops::fmac(w4, 1.6, Ops::fmac(Lam[0], 1.6, m4));
    K[41] = Ops::fmac(w3, 0.8, Ops::fmac(Lam[8], 1.6, Ops::fmac(Lam[0], 0.8, m5)));
    K[42] = Ops::fmac(w4, 0.8, Ops::fmac(Lam[5], 0.8, Ops::fmac(Lam[1], 1.6, m5)));
    K[43] = Ops::fmac(w5, 0.8, Ops::fmac(w1, 0.8, m6));
    K[44] = Ops::fmac(w4, 0.8, Ops::fmac(Lam[8], 0.8, Ops::fmac(Lam[3], 1.6, m5)));
    K[45] = Ops::fmac(Lam[9], 1.6, Ops::fmac(Lam[3], 1.6, Ops::fmac(Lam[0], 1.6, m4)));
    K[46] = Ops::fmac(w8, 0.8, Ops::fmac(w2, 0.8, m6));
    K[47] = Ops::fmac(w7, 0.8, Ops::fmac(Lam[3], 0.8, Ops::fmac(Lam[1], 1.6, m5)));
    K[48] = Ops::fmac(w5, 0.8, Ops::fmac(Lam[9], 0.8, Ops::fmac(Lam[2], 1.6, m5)));
    K[49] = Ops::fmac(w9, 1.6, Ops::fmac(Lam[4], 1.6, m4));
    K[50] = Ops::fmac(w6, 0.8, Ops::fmac(Lam[8], 1.6, Ops::fmac(Lam[4], 0.8, m5)));
    K[51] = Ops::fmac(w9, 0.8, Ops::fmac(Lam[8], 0.8, Ops::fmac(Lam[6], 1.6, m5)));
    K[52] = Ops::fmac(w7, 1.6, Ops::fmac(Lam[4], 1.6, m4));
    K[53] = Ops::fmac(w7, 0.8, Ops::fmac(Lam[8], 0.8, Ops::fmac(Lam[5], 1.6, m5)));
    K[54] = Ops::fmac(Lam[9], 1.6, Ops::fmac(Lam[8], 1.6, Ops::fmac(Lam[7], 1.6, m4)));
  }
  template <class Ops> __device__ __forceinline__ static void mass_upper(const typename Ops::T& vol, typename Ops::T* K) {
    const typename Ops::T m0 = Ops::mulc(vol, 0.014285714285714285);
    const typename Ops::T m1 = Ops::mulc(vol, 0.002380952380952381);
    const typename Ops::T m2 = Ops::mulc(vol, -0.009523809523809525);
    const typename Ops::T m3 = Ops::mulc(vol, -0.014285714285714285);
    const typename Ops::T m4 = Ops::mulc(vol, 0.0761904761904762);
    const typename Ops::T m5 = Ops::mulc(vol, 0.0380952380952381);
    const typename Ops::T m6 = Ops::mulc(vol, 0.01904761904761905);
    K[0] = m0;
    K[1] = m1;
    K[2] = m1;
    K[3] = m1;
    K[4] = m2;
    K[5] = m2;
    K[6] = m2;
    K[7] = m3;
    K[8] = m3;
    K[9] = m3;
    K[10] = m0;
    K[11] = m1;
    K[12] = m1;
    K[13] = m2;
    K[14] = m3;
    K[15] = m3;
    K[16] = m2;
    K[17] = m2;
    K[18] = m3;
    K[19] = m0;
    K[20] = m1;
    K[21] = m3;
    K[22] = m2;
    K[23] = m3;
    K[24] = m2;
    K[25] = m3;
    K[26] = m2;
    K[27] = m0;
    K[28] = m3;
    K[29] = m3;
    K[30] = m2;
    K[31] = m3;
    K[32] = m2;
    K[33] = m2;
    K[34] = m4;
    K[35] = m5;
    K[36] = m5;
    K[37] = m5;
    K[38] = m5;
    K[39] = m6;
    K[40] = m4;
    K[41] = m5;
    K[42] = m5;
    K[43] = m6;
    K[44] = m5;
    K[45] = m4;
    K[46] = m6;
    K[47] = m5;
    K[48] = m5;
    K[49] = m4;
    K[50] = m5;
    K[51] = m5;
    K[52] = m4;
    K[53] = m5;
    K[54] = m4;
  }
  template <class Ops, bool STIFF, bool MASS> __device__ __forceinline__ static void action_upper(const typename Ops::T* Lam, const typename Ops::T& vol, const typename Ops::T* x, typename Ops::T* y) {
    typename Ops::T k;
    if constexpr (STIFF && MASS) {
      const typename Ops::T w0 = Ops::add(Lam[0], Lam[1]);
      const typename Ops::T w1 = Ops::add(Lam[1], Lam[5]);
      const typename Ops::T w2 = Ops::add(Lam[1], Lam[6]);
      const typename Ops::T w3 = Ops::add(Lam[2], Lam[3]);
      const typename Ops::T w4 = Ops::add(Lam[2], Lam[7]);
      const typename Ops::T w5 = Ops::add(Lam[3], Lam[8]);
      const typename Ops::T w6 = Ops::add(Lam[5], Lam[6]);
      const typename Ops::T w7 = Ops::add(Lam[6], Lam[9]);
      const typename Ops::T w8 = Ops::add(Lam[2], Lam[8]);
      const typename Ops::T w9 = Ops::add(Lam[5], Lam[7]);
      const typename Ops::T m0 = Ops::mulc(vol, 0.014285714285714285);
      const typename Ops::T m1 = Ops::mulc(vol, 0.002380952380952381);
      const typename Ops::T m2 = Ops::mulc(vol, -0.009523809523809525);
      const typename Ops::T m3 = Ops::mulc(vol, -0.014285714285714285);
      const typename Ops::T m4 = Ops::mulc(vol, 0.0761904761904762);
      const typename Ops::T m5 = Ops::mulc(vol, 0.0380952380952381);
      const typename Ops::T m6 = Ops::mulc(vol, 0.01904761904761905);
      { k = Ops::fmac(Lam[0], 0.6, m0); y[0] = Ops::mul(k, x[0]); }
      { k = Ops::fmac(Lam[1], -0.2, m1); y[0] = Ops::fma3(k, x[1], y[0]); y[1] = Ops::mul(k, x[0]); }
      { k = Ops::fmac(Lam[2], -0.2, m1); y[0] = Ops::fma3(k, x[2], y[0]); y[2] = Ops::mul(k, x[0]); }
      { k = Ops::fmac(Lam[3], -0.2, m1); y[0] = Ops::fma3(k, x[3], y[0]); y[3] = Ops::mul(k, x[0]); }
      { k = Ops::fmac(Lam[1], 0.6, Ops::fmac(Lam[0], -0.2, m2)); y[0] = Ops::fma3(k, x[4], y[0]); y[4] = Ops::mul(k, x[0]); }
      { k = Ops::fmac(Lam[2], 0.6, Ops::fmac(Lam[0], -0.2, m2)); y[0] = Ops::fma3(k, x[5], y[0]); y[5] = Ops::mul(k, x[0]); }
      { k = Ops::fmac(Lam[3], 0.6, Ops::fmac(Lam[0], -0.2, m2)); y[0] = Ops::fma3(k, x[6], y[0]); y[6] = Ops::mul(k, x[0]); }
      { k = Ops::fmac(Lam[2], -0.2, Ops::fmac(Lam[1], -0.2, m3)); y[0] = Ops::fma3(k, x[7], y[0]); y[7] = Ops::mul(k, x[0]); }
      { k = Ops::fmac(Lam[3], -0.2, Ops::fmac(Lam[1], -0.2, m3)); y[0] = Ops::fma3(k, x[8], y[0]); y[8] = Ops::mul(k, x[0]); }
      { k = Ops::fmac(w3, -0.2, m3); y[0] = Ops::fma3(k, x[9], y[0]); y[9] = Ops::mul(k, x[0]); }
      { k = Ops::fmac(Lam[4], 0.6, m0); y[1] = Ops::fma3(k, x[1], y[1]); }
      { k = Ops::fmac(Lam[5], -0.2, m1); y[1] = Ops::fma3(k, x[2], y[1]); y[2] = Ops::fma3(k, x[1], y[2]); }
      { k = Ops::fmac(Lam[6], -0.2, m1); y[1] = Ops::fma3(k, x[3], y[1]); y[3] = Ops::fma3(k, x[1], y[3]); }
      { k = Ops::fmac(Lam[4], -0.2, Ops::fmac(Lam[1], 0.6, m2)); y[1] = Ops::fma3(k, x[4], y[1]); y[4] = Ops::fma3(k, x[1], y[4]); }
      { k = Ops::fmac(w1, -0.2, m3); y[1] = Ops::fma3(k, x[5], y[1]); y[5] = Ops::fma3(k, x[1], y[5]); }
      { k = Ops::fmac(w2, -0.2, m3); y[1] = Ops::fma3(k, x[6], y[1]); y[6] = Ops::fma3(k, x[1], y[6]); }
      { k = Ops::fmac(Lam[5], 0.6, Ops::fmac(Lam[4], -0.2, m2)); y[1] = Ops::fma3(k, x[7], y[1]); y[7] = Ops::fma3(k, x[1], y[7]); }
      { k = Ops::fmac(Lam[6], 0.6, Ops::fmac(Lam[4], -0.2, m2)); y[1] = Ops::fma3(k, x[8], y[1]); y[8] = Ops::fma3(k, x[1], y[8]); }
      { k = Ops::fmac(w6, -0.2, m3); y[1] = Ops::fma3(k, x[9], y[1]); y[9] = Ops::fma3(k, x[1], y[9]); }
      { k = Ops::fmac(Lam[7], 0.6, m0); y[2] = Ops::fma3(k, x[2], y[2]); }
      { k = Ops::fmac(Lam[8], -0.2, m1); y[2] = Ops::fma3(k, x[3], y[2]); y[3] = Ops::fma3(k, x[2], y[3]); }
      { k = Ops::fmac(Lam[5], -0.2, Ops::fmac(Lam[2], -0.2, m3)); y[2] = Ops::fma3(k, x[4], y[2]); y[4] = Ops::fma3(k, x[2], y[4]); }
      { k = Ops::fmac(Lam[7], -0.2, Ops::fmac(Lam[2], 0.6, m2)); y[2] = Ops::fma3(k, x[5], y[2]); y[5] = Ops::fma3(k, x[2], y[5]); }
      { k = Ops::fmac(w8, -0.2, m3); y[2] = Ops::fma3(k, x[6], y[2]); y[6] = Ops::fma3(k, x[2], y[6]); }
      { k = Ops::fmac(Lam[7], -0.2, Ops::fmac(Lam[5], 0.6, m2)); y[2] = Ops::fma3(k, x[7], y[2]); y[7] = Ops::fma3(k, x[2], y[7]); }
      { k = Ops::fmac(Lam[8], -0.2, Ops::fmac(Lam[5], -0.2, m3)); y[2] = Ops::fma3(k, x[8], y[2]); y[8] = Ops::fma3(k, x[2], y[8]); }
      { k = Ops::fmac(Lam[8], 0.6, Ops::fmac(Lam[7], -0.2, m2)); y[2] = Ops::fma3(k, x[9], y[2]); y[9] = Ops::fma3(k, x[2], y[9]); }
      { k = Ops::fmac(Lam[9], 0.6, m0); y[3] = Ops::fma3(k, x[3], y[3]); }
      { k = Ops::fmac(Lam[6], -0.2, Ops::fmac(Lam[3], -0.2, m3)); y[3] = Ops::fma3(k, x[4], y[3]); y[4] = Ops::fma3(k, x[3], y[4]); }
      { k = Ops::fmac(w5, -0.2, m3); y[3] = Ops::fma3(k, x[5], y[3]); y[5] = Ops::fma3(k, x[3], y[5]); }
      { k = Ops::fmac(Lam[9], -0.2, Ops::fmac(Lam[3], 0.6, m2)); y[3] = Ops::fma3(k, x[6], y[3]); y[6] = Ops::fma3(k, x[3], y[6]); }
      { k = Ops::fmac(Lam[8], -0.2, Ops::fmac(Lam[6], -0.2, m3)); y[3] = Ops::fma3(k, x[7], y[3]); y[7] = Ops::fma3(k, x[3], y[7]); }
      { k = Ops::fmac(Lam[9], -0.2, Ops::fmac(Lam[6], 0.6, m2)); y[3] = Ops::fma3(k, x[8], y[3]); y[8] = Ops::fma3(k, x[3], y[8]); }
      { k = Ops::fmac(Lam[9], -0.2, Ops::fmac(Lam[8], 0.6, m2)); y[3] = Ops::fma3(k, x[9], y[3]); y[9] = Ops::fma3(k, x[3], y[9]); }
      { k = Ops::fmac(w0, 1.6, Ops::fmac(Lam[4], 1.6, m4)); y[4] = Ops::fma3(k, x[4], y[4]); }
      { k = Ops::fmac(w0, 0.8, Ops::fmac(Lam[5], 1.6, Ops::fmac(Lam[2], 0.8, m5))); y[4] = Ops::fma3(k, x[5], y[4]); y[5] = Ops::fma3(k, x[4], y[5]); }
      { k = Ops::fmac(w0, 0.8, Ops::fmac(Lam[6], 1.6, Ops::fmac(Lam[3], 0.8, m5))); y[4] = Ops::fma3(k, x[6], y[4]); y[6] = Ops::fma3(k, x[4], y[6]); }
      { k = Ops::fmac(w1, 0.8, Ops::fmac(Lam[4], 0.8, Ops::fmac(Lam[2], 1.6, m5))); y[4] = Ops::fma3(k, x[7], y[4]); y[7] = Ops::fma3(k, x[4], y[7]); }
      { k = Ops::fmac(w2, 0.8, Ops::fmac(Lam[4], 0.8, Ops::fmac(Lam[3], 1.6, m5))); y[4] = Ops::fma3(k, x[8], y[4]); y[8] = Ops::fma3(k, x[4], y[8]); }
      { k = Ops::fmac(w6, 0.8, Ops::fmac(w3, 0.8, m6)); y[4] = Ops::fma3(k, x[9], y[4]); y[9] = Ops::fma3(k, x[4], y[9]); }
      { k = Ops::fmac(w4, 1.6, Ops::fmac(Lam[0], 1.6, m4)); y[5] = Ops::fma3(k, x[5], y[5]); }
      { k = Ops::fmac(w3, 0.8, Ops::fmac(Lam[8], 1.6, Ops::fmac(Lam[0], 0.8, m5))); y[5] = Ops::fma3(k, x[6], y[5]); y[6] = Ops::fma3(k, x[5], y[6]); }
      { k = Ops::fmac(w4, 0.8, Ops::fmac(Lam[5], 0.8, Ops::fmac(Lam[1], 1.6, m5))); y[5] = Ops::fma3(k, x[7], y[5]); y[7] = Ops::fma3(k, x[5], y[7]); }
      { k = Ops::fmac(w5, 0.8, Ops::fmac(w1, 0.8, m6)); y[5] = Ops::fma3(k, x[8], y[5]); y[8] = Ops::fma3(k, x[5], y[8]); }
      { k = Ops::fmac(w4, 0.8, Ops::fmac(Lam[8], 0.8, Ops::fmac(Lam[3], 1.6, m5))); y[5] = Ops::fma3(k, x[9], y[5]); y[9] = Ops::fma3(k, x[5], y[9]); }
      { k = Ops::fmac(Lam[9], 1.6, Ops::fmac(Lam[3], 1.6, Ops::fmac(Lam[0], 1.6, m4))); y[6] = Ops::fma3(k, x[6], y[6]); }
      { k = Ops::fmac(w8, 0.8, Ops::fmac(w2, 0.8, m6)); y[6] = Ops::fma3(k, x[7], y[6]); y[7] = Ops::fma3(k, x[6], y[7]); }
      { k = Ops::fmac(w7, 0.8, Ops::fmac(Lam[3], 0.8, Ops::fmac(Lam[1], 1.6, m5))); y[6] = Ops::fma3(k, x[8], y[6]); y[8] = Ops::fma3(k, x[6], y[8]); }
      { k = Ops::fmac(w5, 0.8, Ops::fmac(Lam[9], 0.8, Ops::fmac(Lam[2], 1.6, m5))); y[6] = Ops::fma3(k, x[9], y[6]); y[9] = Ops::fma3(k, x[6], y[9]); }
      { k = Ops::fmac(w9, 1.6, Ops::fmac(Lam[4], 1.6, m4)); y[7] = Ops::fma3(k, x[7], y[7]); }
      { k = Ops::fmac(w6, 0.8, Ops::fmac(Lam[8], 1.6, Ops::fmac(Lam[4], 0.8, m5))); y[7] = Ops::fma3(k, x[8], y[7]); y[8] = Ops::fma3(k, x[7], y[8]); }
      { k = Ops::fmac(w9, 0.8, Ops::fmac(Lam[8], 0.8, Ops::fmac(Lam[6], 1.6, m5))); y[7] = Ops::fma3(k, x[9], y[7]); y[9] = Ops::fma3(k, x[7], y[9]); }
      { k = Ops::fmac(w7, 1.6, Ops::fmac(Lam[4], 1.6, m4)); y[8] = Ops::fma3(k, x[8], y[8]); }
      { k = Ops::fmac(w7, 0.8, Ops::fmac(Lam[8], 0.8, Ops::fmac(Lam[5], 1.6, m5))); y[8] = Ops::fma3(k, x[9], y[8]); y[9] = Ops::fma3(k, x[8], y[9]); }
      { k = Ops::fmac(Lam[9], 1.6, Ops::fmac(Lam[8], 1.6, Ops::fmac(Lam[7], 1.6, m4))); y[9] = Ops::fma3(k, x[9], y[9]); }
    }
    else if constexpr (STIFF) {
      const typename Ops::T w0 = Ops::add(Lam[0], Lam[1]);
      const typename Ops::T w1 = Ops::add(Lam[1], Lam[5]);
      const typename Ops::T w2 = Ops::add(Lam[1], Lam[6]);
      const typename Ops::T w3 = Ops::add(Lam[2], Lam[3]);
      const typename Ops::T w4 = Ops::add(Lam[2], Lam[7]);
      const typename Ops::T w5 = Ops::add(Lam[3], Lam[8]);
      const typename Ops::T w6 = Ops::add(Lam[5], Lam[6]);
      const typename Ops::T w7 = Ops::add(Lam[6], Lam[9]);
      const typename Ops::T w8 = Ops::add(Lam[2], Lam[8]);
      const typename Ops::T w9 = Ops::add(Lam[5], Lam[7]);
      { k = Ops::mulc(Lam[0], 0.6); y[0] = Ops::mul(k, x[0]); }
      { k = Ops::mulc(Lam[1], -0.2); y[0] = Ops::fma3(k, x[1], y[0]); y[1] = Ops::mul(k, x[0]); }
      { k = Ops::mulc(Lam[2], -0.2); y[0] = Ops::fma3(k, x[2], y[0]); y[2] = Ops::mul(k, x[0]); }
      { k = Ops::mulc(Lam[3], -0.2); y[0] = Ops::fma3(k, x[3], y[0]); y[3] = Ops::mul(k, x[0]); }
      { k = Ops::fmac(Lam[1], 0.6, Ops::mulc(Lam[0], -0.2)); y[0] = Ops::fma3(k, x[4], y[0]); y[4] = Ops::mul(k, x[0]); }
      { k = Ops::fmac(Lam[2], 0.6, Ops::mulc(Lam[0], -0.2)); y[0] = Ops::fma3(k, x[5], y[0]); y[5] = Ops::mul(k, x[0]); }
      { k = Ops::fmac(Lam[3], 0.6, Ops::mulc(Lam[0], -0.2)); y[0] = Ops::fma3(k, x[6], y[0]); y[6] = Ops::mul(k, x[0]); }
      { k = Ops::fmac(Lam[2], -0.2, Ops::mulc(Lam[1], -0.2)); y[0] = Ops::fma3(k, x[7], y[0]); y[7] = Ops::mul(k, x[0]); }
      { k = Ops::fmac(Lam[3], -0.2, Ops::mulc(Lam[1], -0.2)); y[0] = Ops::fma3(k, x[8], y[0]); y[8] = Ops::mul(k, x[0]); }
      { k = Ops::mulc(w3, -0.2); y[0] = Ops::fma3(k, x[9], y[0]); y[9] = Ops::mul(k, x[0]); }
      { k = Ops::mulc(Lam[4], 0.6); y[1] = Ops::fma3(k, x[1], y[1]); }
      { k = Ops::mulc(Lam[5], -0.2); y[1] = Ops::fma3(k, x[2], y[1]); y[2] = Ops::fma3(k, x[1], y[2]); }
      { k = Ops::mulc(Lam[6], -0.2); y[1] = Ops::fma3(k, x[3], y[1]); y[3] = Ops::fma3(k, x[1], y[3]); }
      { k = Ops::fmac(Lam[4], -0.2, Ops::mulc(Lam[1], 0.6)); y[1] = Ops::fma3(k, x[4], y[1]); y[4] = Ops::fma3(k, x[1], y[4]); }
      { k = Ops::mulc(w1, -0.2); y[1] = Ops::fma3(k, x[5], y[1]); y[5] = Ops::fma3(k, x[1], y[5]); }
      { k = Ops::mulc(w2, -0.2); y[1] = Ops::fma3(k, x[6], y[1]); y[6] = Ops::fma3(k, x[1], y[6]); }
      { k = Ops::fmac(Lam[5], 0.6, Ops::mulc(Lam[4], -0.2)); y[1] = Ops::fma3(k, x[7], y[1]); y[7] = Ops::fma3(k, x[1], y[7]); }
      { k = Ops::fmac(Lam[6], 0.6, Ops::mulc(Lam[4], -0.2)); y[1] = Ops::fma3(k, x[8], y[1]); y[8] = Ops::fma3(k, x[1], y[8]); }
      { k = Ops::mulc(w6, -0.2); y[1] = Ops::fma3(k, x[9], y[1]); y[9] = Ops::fma3(k, x[1], y[9]); }
      { k = Ops::mulc(Lam[7], 0.6); y[2] = Ops::fma3(k, x[2], y[2]); }
      { k = Ops::mulc(Lam[8], -0.2); y[2] = Ops::fma3(k, x[3], y[2]); y[3] = Ops::fma3(k, x[2], y[3]); }
      { k = Ops::fmac(Lam[5], -0.2, Ops::mulc(Lam[2], -0.2)); y[2] = Ops::fma3(k, x[4], y[2]); y[4] = Ops::fma3(k, x[2], y[4]); }
      { k = Ops::fmac(Lam[7], -0.2, Ops::mulc(Lam[2], 0.6)); y[2] = Ops::fma3(k, x[5], y[2]); y[5] = Ops::fma3(k, x[2], y[5]); }
      { k = Ops::mulc(w8, -0.2); y[2] = Ops::fma3(k, x[6], y[2]); y[6] = Ops::fma3(k, x[2], y[6]); }
      { k = Ops::fmac(Lam[7], -0.2, Ops::mulc(Lam[5], 0.6)); y[2] = Ops::fma3(k, x[7], y[2]); y[7] = Ops::fma3(k, x[2], y[7]); }
      { k = Ops::fmac(Lam[8], -0.2, Ops::mulc(Lam[5], -0.2)); y[2] = Ops::fma3(k, x[8], y[2]); y[8] = Ops::fma3(k, x[2], y[8]); }
      { k = Ops::fmac(Lam[8], 0.6, Ops::mulc(Lam[7], -0.2)); y[2] = Ops::fma3(k, x[9], y[2]); y[9] = Ops::fma3(k, x[2], y[9]); }
      { k = Ops::mulc(Lam[9], 0.6); y[3] = Ops::fma3(k, x[3], y[3]); }
      { k = Ops::fmac(Lam[6], -0.2, Ops::mulc(Lam[3], -0.2)); y[3] = Ops::fma3(k, x[4], y[3]); y[4] = Ops::fma3(k, x[3], y[4]); }
      { k = Ops::mulc(w5, -0.2); y[3] = Ops::fma3(k, x[5], y[3]); y[5] = Ops::fma3(k, x[3], y[5]); }
      { k = Ops::fmac(Lam[9], -0.2, Ops::mulc(Lam[3], 0.6)); y[3] = Ops::fma3(k, x[6], y[3]); y[6] = Ops::fma3(k, x[3], y[6]); }
      { k = Ops::fmac(Lam[8], -0.2, Ops::mulc(Lam[6], -0.2)); y[3] = Ops::fma3(k, x[7], y[3]); y[7] = Ops::fma3(k, x[3], y[7]); }
      { k = Ops::fmac(Lam[9], -0.2, Ops::mulc(Lam[6], 0.6)); y[3] = Ops::fma3(k, x[8], y[3]); y[8] = Ops::fma3(k, x[3], y[8]); }
      { k = Ops::fmac(Lam[9], -0.2, Ops::mulc(Lam[8], 0.6)); y[3] = Ops::fma3(k, x[9], y[3]); y[9] = Ops::fma3(k, x[3], y[9]); }
      { k = Ops::fmac(w0, 1.6, Ops::mulc(Lam[4], 1.6)); y[4] = Ops::fma3(k, x[4], y[4]); }
      { k = Ops::fmac(w0, 0.8, Ops::fmac(Lam[5], 1.6, Ops::mulc(Lam[2], 0.8))); y[4] = Ops::fma3(k, x[5], y[4]); y[5] = Ops::fma3(k, x[4], y[5]); }
      { k = Ops::fmac(w0, 0.8, Ops::fmac(Lam[6], 1.6, Ops::mulc(Lam[3], 0.8))); y[4] = Ops::fma3(k, x[6], y[4]); y[6] = Ops::fma3(k, x[4], y[6]); }
      { k = Ops::fmac(w1, 0.8, Ops::fmac(Lam[4], 0.8, Ops::mulc(Lam[2], 1.6))); y[4] = Ops::fma3(k, x[7], y[4]); y[7] = Ops::fma3(k, x[4], y[7]); }
      { k = Ops::fmac(w2, 0.8, Ops::fmac(Lam[4], 0.8, Ops::mulc(Lam[3], 1.6))); y[4] = Ops::fma3(k, x[8], y[4]); y[8] = Ops::fma3(k, x[4], y[8]); }
      { k = Ops::fmac(w6, 0.8, Ops::mulc(w3, 0.8)); y[4] = Ops::fma3(k, x[9], y[4]); y[9] = Ops::fma3(k, x[4], y[9]); }
      { k = Ops::fmac(w4, 1.6, Ops::mulc(Lam[0], 1.6)); y[5] = Ops::fma3(k, x[5], y[5]); }
      { k = Ops::fmac(w3, 0.8, Ops::fmac(Lam[8], 1.6, Ops::mulc(Lam[0], 0.8))); y[5] = Ops::fma3(k, x[6], y[5]); y[6] = Ops::fma3(k, x[5], y[6]); }
      { k = Ops::fmac(w4, 0.8, Ops::fmac(Lam[5], 0.8, Ops::mulc(Lam[1], 1.6))); y[5] = Ops::fma3(k, x[7], y[5]); y[7] = Ops::fma3(k, x[5], y[7]); }
      { k = Ops::fmac(w5, 0.8, Ops::mulc(w1, 0.8)); y[5] = Ops::fma3(k, x[8], y[5]); y[8] = Ops::fma3(k, x[5], y[8]); }
      { k = Ops::fmac(w4, 0.8, Ops::fmac(Lam[8], 0.8, Ops::mulc(Lam[3], 1.6))); y[5] = Ops::fma3(k, x[9], y[5]); y[9] = Ops::fma3(k, x[5], y[9]); }
      { k = Ops::fmac(Lam[9], 1.6, Ops::fmac(Lam[3], 1.6, Ops::mulc(Lam[0], 1.6))); y[6] = Ops::fma3(k, x[6], y[6]); }
      { k = Ops::fmac(w8, 0.8, Ops::mulc(w2, 0.8)); y[6] = Ops::fma3(k, x[7], y[6]); y[7] = Ops::fma3(k, x[6], y[7]); }
      { k = Ops::fmac(w7, 0.8, Ops::fmac(Lam[3], 0.8, Ops::mulc(Lam[1], 1.6))); y[6] = Ops::fma3(k, x[8], y[6]); y[8] = Ops::fma3(k, x[6], y[8]); }
      { k = Ops::fmac(w5, 0.8, Ops::fmac(Lam[9], 0.8, Ops::mulc(Lam[2], 1.6))); y[6] = Ops::fma3(k, x[9], y[6]); y[9] = Ops::fma3(k, x[6], y[9]); }
      { k = Ops::fmac(w9, 1.6, Ops::mulc(Lam[4], 1.6)); y[7] = Ops::fma3(k, x[7], y[7]); }
      { k = Ops::fmac(w6, 0.8, Ops::fmac(Lam[8], 1.6, Ops::mulc(Lam[4], 0.8))); y[7] = Ops::fma3(k, x[8], y[7]); y[8] = Ops::fma3(k, x[7], y[8]); }
      { k = Ops::fmac(w9, 0.8, Ops::fmac(Lam[8], 0.8, Ops::mulc(Lam[6], 1.6))); y[7] = Ops::fma3(k, x[9], y[7]); y[9] = Ops::fma3(k, x[7], y[9]); }
      { k = Ops::fmac(w7, 1.6, Ops::mulc(Lam[4], 1.6)); y[8] = Ops::fma3(k, x[8], y[8]); }
      { k = Ops::fmac(w7, 0.8, Ops::fmac(Lam[8], 0.8, Ops::mulc(Lam[5], 1.6))); y[8] = Ops::fma3(k, x[9], y[8]); y[9] = Ops::fma3(k, x[8], y[9]); }
      { k = Ops::fmac(Lam[9], 1.6, Ops::fmac(Lam[8], 1.6, Ops::mulc(Lam[7], 1.6))); y[9] = Ops::fma3(k, x[9], y[9]); }
    }
    else if constexpr (MASS) {
      const typename Ops::T m0 = Ops::mulc(vol, 0.014285714285714285);
      const typename Ops::T m1 = Ops::mulc(vol, 0.002380952380952381);
      const typename Ops::T m2 = Ops::mulc(vol, -0.009523809523809525);
      const typename Ops::T m3 = Ops::mulc(vol, -0.014285714285714285);
      const typename Ops::T m4 = Ops::mulc(vol, 0.0761904761904762);
      const typename Ops::T m5 = Ops::mulc(vol, 0.0380952380952381);
      const typename Ops::T m6 = Ops::mulc(vol, 0.01904761904761905);
      { k = m0; y[0] = Ops::mul(k, x[0]); }
      { k = m1; y[0] = Ops::fma3(k, x[1], y[0]); y[1] = Ops::mul(k, x[0]); }
      { k = m1; y[0] = Ops::fma3(k, x[2], y[0]); y[2] = Ops::mul(k, x[0]); }
      { k = m1; y[0] = Ops::fma3(k, x[3], y[0]); y[3] = Ops::mul(k, x[0]); }
      { k = m2; y[0] = Ops::fma3(k, x[4], y[0]); y[4] = Ops::mul(k, x[0]); }
      { k = m2; y[0] = Ops::fma3(k, x[5], y[0]); y[5] = Ops::mul(k, x[0]); }
      { k = m2; y[0] = Ops::fma3(k, x[6], y[0]); y[6] = Ops::mul(k, x[0]); }
      { k = m3; y[0] = Ops::fma3(k, x[7], y[0]); y[7] = Ops::mul(k, x[0]); }
      { k = m3; y[0] = Ops::fma3(k, x[8], y[0]); y[8] = Ops::mul(k, x[0]); }
      { k = m3; y[0] = Ops::fma3(k, x[9], y[0]); y[9] = Ops::mul(k, x[0]); }
      { k = m0; y[1] = Ops::fma3(k, x[1], y[1]); }
      { k = m1; y[1] = Ops::fma3(k, x[2], y[1]); y[2] = Ops::fma3(k, x[1], y[2]); }
      { k = m1; y[1] = Ops::fma3(k, x[3], y[1]); y[3] = Ops::fma3(k, x[1], y[3]); }
      { k = m2; y[1] = Ops::fma3(k, x[4], y[1]); y[4] = Ops::fma3(k, x[1], y[4]); }
      { k = m3; y[1] = Ops::fma3(k, x[5], y[1]); y[5] = Ops::fma3(k, x[1], y[5]); }
      { k = m3; y[1] = Ops::fma3(k, x[6], y[1]); y[6] = Ops::fma3(k, x[1], y[6]); }
      { k = m2; y[1] = Ops::fma3(k, x[7], y[1]); y[7] = Ops::fma3(k, x[1], y[7]); }
      { k = m2; y[1] = Ops::fma3(k, x[8], y[1]); y[8] = Ops::fma3(k, x[1], y[8]); }
      { k = m3; y[1] = Ops::fma3(k, x[9], y[1]); y[9] = Ops::fma3(k, x[1], y[9]); }
      { k = m0; y[2] = Ops::fma3(k, x[2], y[2]); }
      { k = m1; y[2] = Ops::fma3(k, x[3], y[2]); y[3] = Ops::fma3(k, x[2], y[3]); }
      { k = m3; y[2] = Ops::fma3(k, x[4], y[2]); y[4] = Ops::fma3(k, x[2], y[4]); }
      { k = m2; y[2] = Ops::fma3(k, x[5], y[2]); y[5] = Ops::fma3(k, x[2], y[5]); }
      { k = m3; y[2] = Ops::fma3(k, x[6], y[2]); y[6] = Ops::fma3(k, x[2], y[6]); }
      { k = m2; y[2] = Ops::fma3(k, x[7], y[2]); y[7] = Ops::fma3(k, x[2], y[7]); }
      { k = m3; y[2] = Ops::fma3(k, x[8], y[2]); y[8] = Ops::fma3(k, x[2], y[8]); }
      { k = m2; y[2] = Ops::fma3(k, x[9], y[2]); y[9] = Ops::fma3(k, x[2], y[9]); }
      { k = m0; y[3] = Ops::fma3(k, x[3], y[3]); }
      { k = m3; y[3] = Ops::fma3(k, x[4], y[3]); y[4] = Ops::fma3(k, x[3], y[4]); }
      { k = m3; y[3] = Ops::fma3(k, x[5], y[3]); y[5] = Ops::fma3(k, x[3], y[5]); }
      { k = m2; y[3] = Ops::fma3(k, x[6], y[3]); y[6] = Ops::fma3(k, x[3], y[6]); }
      { k = m3; y[3] = Ops::fma3(k, x[7], y[3]); y[7] = Ops::fma3(k, x[3], y[7]); }
      { k = m2; y[3] = Ops::fma3(k, x[8], y[3]); y[8] = Ops::fma3(k, x[3], y[8]); }
      { k = m2; y[3] = Ops::fma3(k, x[9], y[3]); y[9] = Ops::fma3(k, x[3], y[9]); }
      { k = m4; y[4] = Ops::fma3(k, x[4], y[4]); }
      { k = m5; y[4] = Ops::fma3(k, x[5], y[4]); y[5] = Ops::fma3(k, x[4], y[5]); }
      { k = m5; y[4] = Ops::fma3(k, x[6], y[4]); y[6] = Ops::fma3(k, x[4], y[6]); }
      { k = m5; y[4] = Ops::fma3(k, x[7], y[4]); y[7] = Ops::fma3(k, x[4], y[7]); }
      { k = m5; y[4] = Ops::fma3(k, x[8], y[4]); y[8] = Ops::fma3(k, x[4], y[8]); }
      { k = m6; y[4] = Ops::fma3(k, x[9], y[4]); y[9] = Ops::fma3(k, x[4], y[9]); }
      { k = m4; y[5] = Ops::fma3(k, x[5], y[5]); }
      { k = m5; y[5] = Ops::fma3(k, x[6], y[5]); y[6] = Ops::fma3(k, x[5], y[6]); }
      { k = m5; y[5] = Ops::fma3(k, x[7], y[5]); y[7] = Ops::fma3(k, x[5], y[7]); }
      { k = m6; y[5] = Ops::fma3(k, x[8], y[5]); y[8] = Ops::fma3(k, x[5], y[8]); }
      { k = m5; y[5] = Ops::fma3(k, x[9], y[5]); y[9] = Ops::fma3(k, x[5], y[9]); }
      { k = m4; y[6] = Ops::fma3(k, x[6], y[6]); }
      { k = m6; y[6] = Ops::fma3(k, x[7], y[6]); y[7] = Ops::fma3(k, x[6], y[7]); }
      { k = m5; y[6] = Ops::fma3(k, x[8], y[6]); y[8] = Ops::fma3(k, x[6], y[8]); }
      { k = m5; y[6] = Ops::fma3(k, x[9], y[6]); y[9] = Ops::fma3(k, x[6], y[9]); }
      { k = m4; y[7] = Ops::fma3(k, x[7], y[7]); }
      { k = m5; y[7] = Ops::fma3(k, x[8], y[7]); y[8] = Ops::fma3(k, x[7], y[8]); }
      { k = m5; y[7] = Ops::fma3(k, x[9], y[7]); y[9] = Ops::fma3(k, x[7], y[9]); }
      { k = m4; y[8] = Ops::fma3(k, x[8], y[8]); }
      { k = m5; y[8] = Ops::fma3(k, x[9], y[8]); y[9] = Ops::fma3(k, x[8], y[9]); }
      { k = m4; y[9] = Ops::fma3(k, x[9], y[9]); }
    }
  }
  __host__ __device__ static constexpr int upper_index(int i, int j) {
    return i <= j ? i * 10 - (i * (i - 1)) / 2 + (j - i) : j * 10 - (j * (j - 1)) / 2 + (i - j);
  }
};

// ---- P3 Lagrange on the tetrahedron (20 nodes) ----
template <> struct Elem<3, 3> {
  static constexpr int ND = 20;
  static constexpr int NUP = 210;
  static constexpr int NLAM = 10;
  static constexpr int STIFF_TERMS = 784;
  // K[u] for u over the upper triangle (i <= j), row-major; Lam[k] over pairs (m <= n)
  static constexpr int STIFF_OPS = 490;  // after rewriting
  template <class Ops> __device__ __forceinline__ static void stiffness_upper(const typename Ops::T* Lam, typename Ops::T* K) {
    const typename Ops::T w0 = Ops::add(Lam[1], Lam[2]);
    const typename Ops::T w1 = Ops::add(Lam[3], Lam[6]);
    const typename Ops::T w2 = Ops::add(Lam[5], Lam[8]);
    const typename Ops::T w3 = Ops::add(Lam[0], Lam[3]);
    const typename Ops::T w4 = Ops::add(Lam[1], Lam[4]);
    const typename Ops::T w5 = Ops::add(Lam[2], Lam[7]);
    const typename Ops::T w6 = Ops::add(Lam[8], Lam[9]);
    const typename Ops::T w7 = Ops::add(Lam[5], Lam[6]);
    const typename Ops::T w8 = Ops::add(Lam[1], Lam[3]);
    const typename Ops::T w9 = Ops::add(Lam[2], Lam[5]);
    const typename Ops::T w10 = Ops::add(Lam[6], Lam[8]);
    const typename Ops::T w11 = Ops::add(Lam[1], Lam[5]);
    const typename Ops::T w12 = Ops::add(Lam[1], Lam[6]);
    const typename Ops::T w13 = Ops::add(Lam[2], Lam[3]);
    const typename Ops::T w14 = Ops::add(Lam[2], Lam[8]);
    const typename Ops::T w15 = Ops::add(Lam[3], Lam[8]);
    const typename Ops::T w16 = Ops::add(Lam[0], w0);
    const typename Ops::T w17 = Ops::add(Lam[4], Lam[5]);
    const typename Ops::T w18 = Ops::add(Lam[4], Lam[6]);
    const typename Ops::T w19 = Ops::add(Lam[7], w2);
    const typename Ops::T w20 = Ops::add(Lam[9], w1);
    const typename Ops::T w21 = Ops::add(Lam[0], Lam[1]);
    const typename Ops::T w22 = Ops::add(Lam[0], Lam[2]);
    const typename Ops::T w23 = Ops::add(Lam[3], Lam[9]);
    const typename Ops::T w24 = Ops::add(Lam[5], Lam[7]);
    const typename Ops::T w25 = Ops::add(Lam[6], Lam[9]);
    const typename Ops::T w26 = Ops::add(Lam[7], Lam[8]);
    const typename Ops::T w27 = Ops::add(w0, w3);
    const typename Ops::T w28 = Ops::add(w0, w10);
    const typename Ops::T w29 = Ops::add(w1, w6);
    const typename Ops::T w30 = Ops::add(w1, w9);
    const typename Ops::T w31 = Ops::add(w2, w5);
    const typename Ops::T w32 = Ops::add(w2, w8);
    const typename Ops::T w33 = Ops::add(Lam[1], w3);
    const typename Ops::T w34 = Ops::add(Lam[2], w3);
    const typename Ops::T w35 = Ops::add(Lam[3], w6);
    const typename Ops::T w36 = Ops::add(Lam[4], w7);
    const typename Ops::T w37 = Ops::add(Lam[5], w4);
    const typename Ops::T w38 = Ops::add(Lam[5], w5);
    const typename Ops::T w39 = Ops::add(Lam[6], w4);
    const typename Ops::T w40 = Ops::add(Lam[6], w6);
    const typename Ops::T w41 = Ops::add(Lam[8], w5);
    const typename Ops::T w42 = Ops::add(w4, w7);
    const typename Ops::T w43 = Ops::fmac(Lam[1], -5.0, Lam[0]);
    const typename Ops::T w44 = Ops::fmac(Lam[2], -5.0, Lam[0]);
    const typename Ops::T w45 = Ops::fmac(Lam[3], -5.0, Lam[0]);
    const typename Ops::T w46 = Ops::fmac(Lam[4], -0.2, Lam[1]);
    const typename Ops::T w47 = Ops::fmac(w20, 0.5, Lam[1]);
    const typename Ops::T w48 = Ops::fmac(Lam[7], -0.2, Lam[2]);
    const typename Ops::T w49 = Ops::fmac(Lam[9], -0.2, Lam[3]);
    const typename Ops::T w50 = Ops::fmac(Lam[5], -5.0, Lam[4]);
    const typename Ops::T w51 = Ops::fmac(Lam[6], -5.0, Lam[4]);
    const typename Ops::T w52 = Ops::fmac(Lam[7], -0.2, Lam[5]);
    const typename Ops::T w53 = Ops::fmac(w16, 0.5, Lam[5]);
    const typename Ops::T w54 = Ops::fmac(Lam[9], -0.2, Lam[6]);
    const typename Ops::T w55 = Ops::fmac(w19, 0.5, Lam[6]);
    const typename Ops::T w56 = Ops::fmac(Lam[8], -5.0, Lam[7]);
    const typename Ops::T w57 = Ops::fmac(Lam[9], -0.2, Lam[8]);
    const typename Ops::T w58 = Ops::add(w4, w20);
    const typename Ops::T w59 = Ops::add(w16, w17);
    const typename Ops::T w60 = Ops::add(w18, w19);
    K[0] = Ops::mulc(Lam[0], 0.35714285714285715);
    K[1] = Ops::mulc(Lam[1], 0.06785714285714285);
    K[2] = Ops::mulc(Lam[2], 0.06785714285714285);
    K[3] = Ops::mulc(Lam[3], 0.06785714285714285);
    K[4] = Ops::fmac(Lam[1], 0.36964285714285716, Ops::mulc(Lam[0], -0.20892857142857144));
    K[5] = Ops::fmac(Lam[1], -0.20892857142857144, Ops::mulc(Lam[0], 0.08035714285714286));
    K[6] = Ops::fmac(Lam[2], 0.36964285714285716, Ops::mulc(Lam[0], -0.20892857142857144));
    K[7] = Ops::fmac(Lam[2], -0.20892857142857144, Ops::mulc(Lam[0], 0.08035714285714286));
    K[8] = Ops::fmac(Lam[3], 0.36964285714285716, Ops::mulc(Lam[0], -0.20892857142857144));
    K[9] = Ops::fmac(Lam[3], -0.20892857142857144, Ops::mulc(Lam[0], 0.08035714285714286));
    K[10] = Ops::mulc(w0, 0.08035714285714286);
    K[11] = Ops::mulc(w0, 0.08035714285714286);
    K[12] = Ops::mulc(w8, 0.08035714285714286);
    K[13] = Ops::mulc(w8, 0.08035714285714286);
    K[14] = Ops::mulc(w13, 0.08035714285714286);
    K[15] = Ops::mulc(w13, 0.08035714285714286);
    K[16] = Ops::fmac(w0, -0.09642857142857143, Ops::mulc(Lam[0], 0.19285714285714287));
    K[17] = Ops::fmac(w8, -0.09642857142857143, Ops::mulc(Lam[0], 0.19285714285714287));
    K[18] = Ops::fmac(w13, -0.09642857142857143, Ops::mulc(Lam[0], 0.19285714285714287));
    K[19] = Ops::fmac(w0, 0.19285714285714287, Ops::mulc(Lam[3], 0.19285714285714287));
    K[20] = Ops::mulc(Lam[4], 0.35714285714285715);
    K[21] = Ops::mulc(Lam[5], 0.06785714285714285);
    K[22] = Ops::mulc(Lam[6], 0.06785714285714285);
    K[23] = Ops::fmac(Lam[4], 0.08035714285714286, Ops::mulc(Lam[1], -0.20892857142857144));
    K[24] = Ops::fmac(Lam[4], -0.20892857142857144, Ops::mulc(Lam[1], 0.36964285714285716));
    K[25] = Ops::mulc(w11, 0.08035714285714286);
    K[26] = Ops::mulc(w11, 0.08035714285714286);
    K[27] = Ops::mulc(w12, 0.08035714285714286);
    K[28] = Ops::mulc(w12, 0.08035714285714286);
    K[29] = Ops::fmac(Lam[5], 0.36964285714285716, Ops::mulc(Lam[4], -0.20892857142857144));
    K[30] = Ops::fmac(Lam[5], -0.20892857142857144, Ops::mulc(Lam[4], 0.08035714285714286));
    K[31] = Ops::fmac(Lam[6], 0.36964285714285716, Ops::mulc(Lam[4], -0.20892857142857144));
    K[32] = Ops::fmac(Lam[6], -0.20892857142857144, Ops::mulc(Lam[4], 0.08035714285714286));
    K[33] = Ops::mulc(w7, 0.08035714285714286);
    K[34] = Ops::mulc(w7, 0.08035714285714286);
    K[35] = Ops::fmac(w11, -0.09642857142857143, Ops::mulc(Lam[4], 0.19285714285714287));
    K[36] = Ops::fmac(w12, -0.09642857142857143, Ops::mulc(Lam[4], 0.19285714285714287));
    K[37] = Ops::fmac(w7, 0.19285714285714287, Ops::mulc(Lam[1], 0.19285714285714287));
    K[38] = Ops::fmac(w7, -0.09642857142857143, Ops::mulc(Lam[4], 0.19285714285714287));
    K[39] = Ops::mulc(Lam[7], 0.35714285714285715);
    K[40] = Ops::mulc(Lam[8], 0.06785714285714285);
    K[41] = Ops::mulc(w9, 0.08035714285714286);
    K[42] = Ops::mulc(w9, 0.08035714285714286);
    K[43] = Ops::fmac(Lam[7], 0.08035714285714286, Ops::mulc(Lam[2], -0.20892857142857144));
    K[44] = Ops::fmac(Lam[7], -0.20892857142857144, Ops::mulc(Lam[2], 0.36964285714285716));
    K[45] = Ops::mulc(w14, 0.08035714285714286);
    K[46] = Ops::mulc(w14, 0.08035714285714286);
    K[47] = Ops::fmac(Lam[7], 0.08035714285714286, Ops::mulc(Lam[5], -0.20892857142857144));
    K[48] = Ops::fmac(Lam[7], -0.20892857142857144, Ops::mulc(Lam[5], 0.36964285714285716));
    K[49] = Ops::mulc(w2, 0.08035714285714286);
    K[50] = Ops::mulc(w2, 0.08035714285714286);
    K[51] = Ops::fmac(Lam[8], 0.36964285714285716, Ops::mulc(Lam[7], -0.20892857142857144));
    K[52] = Ops::fmac(Lam[8], -0.20892857142857144, Ops::mulc(Lam[7], 0.08035714285714286));
    K[53] = Ops::fmac(w9, -0.09642857142857143, Ops::mulc(Lam[7], 0.19285714285714287));
    K[54] = Ops::fmac(w2, 0.19285714285714287, Ops::mulc(Lam[2], 0.19285714285714287));
    K[55] = Ops::fmac(w14, -0.09642857142857143, Ops::mulc(Lam[7], 0.19285714285714287));
    K[56] = Ops::fmac(w2, -0.09642857142857143, Ops::mulc(Lam[7], 0.19285714285714287));
    K[57] = Ops::mulc(Lam[9], 0.35714285714285715);
    K[58] = Ops::mulc(w1, 0.08035714285714286);
    K[59] = Ops::mulc(w1, 0.08035714285714286);
    K[60] = Ops::mulc(w15, 0.08035714285714286);
    K[61] = Ops::mulc(w15, 0.08035714285714286);
    K[62] = Ops::fmac(Lam[9], 0.08035714285714286, Ops::mulc(Lam[3], -0.20892857142857144));
    K[63] = Ops::fmac(Lam[9], -0.20892857142857144, Ops::mulc(Lam[3], 0.36964285714285716));
    K[64] = Ops::mulc(w10, 0.08035714285714286);
    K[65] = Ops::mulc(w10, 0.08035714285714286);
    K[66] = Ops::fmac(Lam[9], 0.08035714285714286, Ops::mulc(Lam[6], -0.20892857142857144));
    K[67] = Ops::fmac(Lam[9], -0.20892857142857144, Ops::mulc(Lam[6], 0.36964285714285716));
    K[68] = Ops::fmac(Lam[9], 0.08035714285714286, Ops::mulc(Lam[8], -0.20892857142857144));
    K[69] = Ops::fmac(Lam[9], -0.20892857142857144, Ops::mulc(Lam[8], 0.36964285714285716));
    K[70] = Ops::fmac(w1, 0.19285714285714287, Ops::mulc(Lam[8], 0.19285714285714287));
    K[71] = Ops::fmac(w1, -0.09642857142857143, Ops::mulc(Lam[9], 0.19285714285714287));
    K[72] = Ops::fmac(w15, -0.09642857142857143, Ops::mulc(Lam[9], 0.19285714285714287));
    K[73] = Ops::fmac(w10, -0.09642857142857143, Ops::mulc(Lam[9], 0.19285714285714287));
    K[74] = Ops::fmac(w4, 1.1571428571428573, Ops::mulc(Lam[0], 1.4464285714285714));
    K[75] = Ops::fmac(Lam[4], -0.43392857142857144, Ops::fmac(Lam[1], 0.2892857142857143, Ops::mulc(Lam[0], -0.43392857142857144)));
    K[76] = Ops::fmac(w0, 0.5785714285714286, Ops::fmac(Lam[5], 1.1571428571428573, Ops::mulc(Lam[0], 0.7232142857142857)));
    K[77] = Ops::fmac(w21, -0.14464285714285716, Ops::fmac(Lam[5], -0.43392857142857144, Ops::mulc(Lam[2], -0.2892857142857143)));
    K[78] = Ops::fmac(w8, 0.5785714285714286, Ops::fmac(Lam[6], 1.1571428571428573, Ops::mulc(Lam[0], 0.7232142857142857)));
    K[79] = Ops::fmac(w21, -0.14464285714285716, Ops::fmac(Lam[6], -0.43392857142857144, Ops::mulc(Lam[3], -0.2892857142857143)));
    K[80] = Ops::fmac(w17, -0.14464285714285716, Ops::fmac(Lam[2], -0.43392857142857144, Ops::mulc(Lam[1], -0.2892857142857143)));
    K[81] = Ops::fmac(w37, -0.14464285714285716, Ops::mulc(Lam[2], -0.2892857142857143));
    K[82] = Ops::fmac(w18, -0.14464285714285716, Ops::fmac(Lam[3], -0.43392857142857144, Ops::mulc(Lam[1], -0.2892857142857143)));
    K[83] = Ops::fmac(w39, -0.14464285714285716, Ops::mulc(Lam[3], -0.2892857142857143));
    K[84] = Ops::mulc(w30, -0.14464285714285716);
    K[85] = Ops::mulc(w30, -0.14464285714285716);
    K[86] = Ops::fmac(w44, -0.2892857142857143, Ops::mulc(w37, 0.5785714285714286));
    K[87] = Ops::fmac(w45, -0.2892857142857143, Ops::mulc(w39, 0.5785714285714286));
    K[88] = Ops::fmac(w21, -0.14464285714285716, Ops::fmac(w13, 0.7232142857142857, Ops::mulc(w7, 0.5785714285714286)));
    K[89] = Ops::fmac(w42, -0.14464285714285716, Ops::mulc(w13, -0.2892857142857143));
    K[90] = Ops::fmac(w21, 1.1571428571428573, Ops::mulc(Lam[4], 1.4464285714285714));
    K[91] = Ops::fmac(w22, -0.14464285714285716, Ops::fmac(Lam[5], -0.43392857142857144, Ops::mulc(Lam[1], -0.2892857142857143)));
    K[92] = Ops::mulc(w53, -0.2892857142857143);
    K[93] = Ops::fmac(w3, -0.14464285714285716, Ops::fmac(Lam[6], -0.43392857142857144, Ops::mulc(Lam[1], -0.2892857142857143)));
    K[94] = Ops::fmac(w33, -0.14464285714285716, Ops::mulc(Lam[6], -0.2892857142857143));
    K[95] = Ops::fmac(w11, 0.5785714285714286, Ops::fmac(Lam[4], 0.7232142857142857, Ops::mulc(Lam[2], 1.1571428571428573)));
    K[96] = Ops::fmac(w4, -0.14464285714285716, Ops::fmac(Lam[5], -0.2892857142857143, Ops::mulc(Lam[2], -0.43392857142857144)));
    K[97] = Ops::fmac(w12, 0.5785714285714286, Ops::fmac(Lam[4], 0.7232142857142857, Ops::mulc(Lam[3], 1.1571428571428573)));
    K[98] = Ops::fmac(w4, -0.14464285714285716, Ops::fmac(Lam[6], -0.2892857142857143, Ops::mulc(Lam[3], -0.43392857142857144)));
    K[99] = Ops::mulc(w30, -0.14464285714285716);
    K[100] = Ops::mulc(w30, -0.14464285714285716);
    K[101] = Ops::fmac(w50, -0.2892857142857143, Ops::mulc(w16, 0.5785714285714286));
    K[102] = Ops::fmac(w51, -0.2892857142857143, Ops::mulc(w33, 0.5785714285714286));
    K[103] = Ops::fmac(w27, -0.14464285714285716, Ops::mulc(w7, -0.2892857142857143));
    K[104] = Ops::fmac(w13, 0.5785714285714286, Ops::fmac(w7, 0.7232142857142857, Ops::mulc(w4, -0.14464285714285716)));
    K[105] = Ops::fmac(w5, 1.1571428571428573, Ops::mulc(Lam[0], 1.4464285714285714));
    K[106] = Ops::fmac(Lam[7], -0.43392857142857144, Ops::fmac(Lam[2], 0.2892857142857143, Ops::mulc(Lam[0], -0.43392857142857144)));
    K[107] = Ops::fmac(w13, 0.5785714285714286, Ops::fmac(Lam[8], 1.1571428571428573, Ops::mulc(Lam[0], 0.7232142857142857)));
    K[108] = Ops::fmac(w22, -0.14464285714285716, Ops::fmac(Lam[8], -0.43392857142857144, Ops::mulc(Lam[3], -0.2892857142857143)));
    K[109] = Ops::fmac(w38, -0.14464285714285716, Ops::mulc(Lam[1], -0.2892857142857143));
    K[110] = Ops::fmac(w24, -0.14464285714285716, Ops::fmac(Lam[2], -0.2892857142857143, Ops::mulc(Lam[1], -0.43392857142857144)));
    K[111] = Ops::mulc(w32, -0.14464285714285716);
    K[112] = Ops::mulc(w32, -0.14464285714285716);
    K[113] = Ops::fmac(w26, -0.14464285714285716, Ops::fmac(Lam[3], -0.43392857142857144, Ops::mulc(Lam[2], -0.2892857142857143)));
    K[114] = Ops::fmac(w41, -0.14464285714285716, Ops::mulc(Lam[3], -0.2892857142857143));
    K[115] = Ops::fmac(w43, -0.2892857142857143, Ops::mulc(w38, 0.5785714285714286));
    K[116] = Ops::fmac(w22, -0.14464285714285716, Ops::fmac(w8, 0.7232142857142857, Ops::mulc(w2, 0.5785714285714286)));
    K[117] = Ops::fmac(w45, -0.2892857142857143, Ops::mulc(w41, 0.5785714285714286));
    K[118] = Ops::fmac(w31, -0.14464285714285716, Ops::mulc(w8, -0.2892857142857143));
    K[119] = Ops::fmac(w22, 1.1571428571428573, Ops::mulc(Lam[7], 1.4464285714285714));
    K[120] = Ops::fmac(w3, -0.14464285714285716, Ops::fmac(Lam[8], -0.43392857142857144, Ops::mulc(Lam[2], -0.2892857142857143)));
    K[121] = Ops::fmac(w34, -0.14464285714285716, Ops::mulc(Lam[8], -0.2892857142857143));
    K[122] = Ops::fmac(w5, -0.14464285714285716, Ops::fmac(Lam[5], -0.2892857142857143, Ops::mulc(Lam[1], -0.43392857142857144)));
    K[123] = Ops::fmac(w9, 0.5785714285714286, Ops::fmac(Lam[7], 0.7232142857142857, Ops::mulc(Lam[1], 1.1571428571428573)));
    K[124] = Ops::mulc(w32, -0.14464285714285716);
    K[125] = Ops::mulc(w32, -0.14464285714285716);
    K[126] = Ops::fmac(w14, 0.5785714285714286, Ops::fmac(Lam[7], 0.7232142857142857, Ops::mulc(Lam[3], 1.1571428571428573)));
    K[127] = Ops::fmac(w5, -0.14464285714285716, Ops::fmac(Lam[8], -0.2892857142857143, Ops::mulc(Lam[3], -0.43392857142857144)));
    K[128] = Ops::fmac(w52, 1.4464285714285714, Ops::mulc(w16, 0.5785714285714286));
    K[129] = Ops::fmac(w27, -0.14464285714285716, Ops::mulc(w2, -0.2892857142857143));
    K[130] = Ops::fmac(w56, -0.2892857142857143, Ops::mulc(w34, 0.5785714285714286));
    K[131] = Ops::fmac(w8, 0.5785714285714286, Ops::fmac(w5, -0.14464285714285716, Ops::mulc(w2, 0.7232142857142857)));
    K[132] = Ops::fmac(w23, 1.1571428571428573, Ops::mulc(Lam[0], 1.4464285714285714));
    K[133] = Ops::fmac(Lam[9], -0.43392857142857144, Ops::fmac(Lam[3], 0.2892857142857143, Ops::mulc(Lam[0], -0.43392857142857144)));
    K[134] = Ops::mulc(w28, -0.14464285714285716);
    K[135] = Ops::mulc(w28, -0.14464285714285716);
    K[136] = Ops::mulc(w47, -0.2892857142857143);
    K[137] = Ops::fmac(w25, -0.14464285714285716, Ops::fmac(Lam[3], -0.2892857142857143, Ops::mulc(Lam[1], -0.43392857142857144)));
    K[138] = Ops::fmac(w35, -0.14464285714285716, Ops::mulc(Lam[2], -0.2892857142857143));
    K[139] = Ops::fmac(w6, -0.14464285714285716, Ops::fmac(Lam[3], -0.2892857142857143, Ops::mulc(Lam[2], -0.43392857142857144)));
    K[140] = Ops::fmac(w10, 0.5785714285714286, Ops::fmac(w3, -0.14464285714285716, Ops::mulc(w0, 0.7232142857142857)));
    K[141] = Ops::fmac(w43, -0.2892857142857143, Ops::mulc(w20, 0.5785714285714286));
    K[142] = Ops::fmac(w44, -0.2892857142857143, Ops::mulc(w35, 0.5785714285714286));
    K[143] = Ops::fmac(w29, -0.14464285714285716, Ops::mulc(w0, -0.2892857142857143));
    K[144] = Ops::fmac(w3, 1.1571428571428573, Ops::mulc(Lam[9], 1.4464285714285714));
    K[145] = Ops::mulc(w28, -0.14464285714285716);
    K[146] = Ops::mulc(w28, -0.14464285714285716);
    K[147] = Ops::fmac(w23, -0.14464285714285716, Ops::fmac(Lam[6], -0.2892857142857143, Ops::mulc(Lam[1], -0.43392857142857144)));
    K[148] = Ops::fmac(w1, 0.5785714285714286, Ops::fmac(Lam[9], 0.7232142857142857, Ops::mulc(Lam[1], 1.1571428571428573)));
    K[149] = Ops::fmac(w23, -0.14464285714285716, Ops::fmac(Lam[8], -0.2892857142857143, Ops::mulc(Lam[2], -0.43392857142857144)));
    K[150] = Ops::fmac(w15, 0.5785714285714286, Ops::fmac(Lam[9], 0.7232142857142857, Ops::mulc(Lam[2], 1.1571428571428573)));
    K[151] = Ops::fmac(w27, -0.14464285714285716, Ops::mulc(w10, -0.2892857142857143));
    K[152] = Ops::fmac(w54, 1.4464285714285714, Ops::mulc(w33, 0.5785714285714286));
    K[153] = Ops::fmac(w57, 1.4464285714285714, Ops::mulc(w34, 0.5785714285714286));
    K[154] = Ops::fmac(w23, -0.14464285714285716, Ops::fmac(w10, 0.7232142857142857, Ops::mulc(w0, 0.5785714285714286)));
    K[155] = Ops::fmac(w24, 1.1571428571428573, Ops::mulc(Lam[4], 1.4464285714285714));
    K[156] = Ops::fmac(Lam[7], -0.43392857142857144, Ops::fmac(Lam[5], 0.2892857142857143, Ops::mulc(Lam[4], -0.43392857142857144)));
    K[157] = Ops::fmac(w7, 0.5785714285714286, Ops::fmac(Lam[8], 1.1571428571428573, Ops::mulc(Lam[4], 0.7232142857142857)));
    K[158] = Ops::fmac(w17, -0.14464285714285716, Ops::fmac(Lam[8], -0.43392857142857144, Ops::mulc(Lam[6], -0.2892857142857143)));
    K[159] = Ops::fmac(w26, -0.14464285714285716, Ops::fmac(Lam[6], -0.43392857142857144, Ops::mulc(Lam[5], -0.2892857142857143)));
    K[160] = Ops::mulc(w55, -0.2892857142857143);
    K[161] = Ops::fmac(w46, 1.4464285714285714, Ops::mulc(w38, 0.5785714285714286));
    K[162] = Ops::fmac(w17, -0.14464285714285716, Ops::fmac(w14, 0.5785714285714286, Ops::mulc(w12, 0.7232142857142857)));
    K[163] = Ops::fmac(w31, -0.14464285714285716, Ops::mulc(w12, -0.2892857142857143));
    K[164] = Ops::fmac(w51, -0.2892857142857143, Ops::mulc(w19, 0.5785714285714286));
    K[165] = Ops::fmac(w17, 1.1571428571428573, Ops::mulc(Lam[7], 1.4464285714285714));
    K[166] = Ops::fmac(w18, -0.14464285714285716, Ops::fmac(Lam[8], -0.43392857142857144, Ops::mulc(Lam[5], -0.2892857142857143)));
    K[167] = Ops::fmac(w36, -0.14464285714285716, Ops::mulc(Lam[8], -0.2892857142857143));
    K[168] = Ops::fmac(w2, 0.5785714285714286, Ops::fmac(Lam[7], 0.7232142857142857, Ops::mulc(Lam[6], 1.1571428571428573)));
    K[169] = Ops::fmac(w24, -0.14464285714285716, Ops::fmac(Lam[8], -0.2892857142857143, Ops::mulc(Lam[6], -0.43392857142857144)));
    K[170] = Ops::fmac(w48, 1.4464285714285714, Ops::mulc(w37, 0.5785714285714286));
    K[171] = Ops::fmac(w42, -0.14464285714285716, Ops::mulc(w14, -0.2892857142857143));
    K[172] = Ops::fmac(w24, -0.14464285714285716, Ops::fmac(w14, 0.7232142857142857, Ops::mulc(w12, 0.5785714285714286)));
    K[173] = Ops::fmac(w56, -0.2892857142857143, Ops::mulc(w36, 0.5785714285714286));
    K[174] = Ops::fmac(w25, 1.1571428571428573, Ops::mulc(Lam[4], 1.4464285714285714));
    K[175] = Ops::fmac(Lam[9], -0.43392857142857144, Ops::fmac(Lam[6], 0.2892857142857143, Ops::mulc(Lam[4], -0.43392857142857144)));
    K[176] = Ops::fmac(w40, -0.14464285714285716, Ops::mulc(Lam[5], -0.2892857142857143));
    K[177] = Ops::fmac(w6, -0.14464285714285716, Ops::fmac(Lam[6], -0.2892857142857143, Ops::mulc(Lam[5], -0.43392857142857144)));
    K[178] = Ops::fmac(w18, -0.14464285714285716, Ops::fmac(w15, 0.5785714285714286, Ops::mulc(w11, 0.7232142857142857)));
    K[179] = Ops::fmac(w46, 1.4464285714285714, Ops::mulc(w20, 0.5785714285714286));
    K[180] = Ops::fmac(w29, -0.14464285714285716, Ops::mulc(w11, -0.2892857142857143));
    K[181] = Ops::fmac(w50, -0.2892857142857143, Ops::mulc(w40, 0.5785714285714286));
    K[182] = Ops::fmac(w18, 1.1571428571428573, Ops::mulc(Lam[9], 1.4464285714285714));
    K[183] = Ops::fmac(w25, -0.14464285714285716, Ops::fmac(Lam[8], -0.2892857142857143, Ops::mulc(Lam[5], -0.43392857142857144)));
    K[184] = Ops::fmac(w10, 0.5785714285714286, Ops::fmac(Lam[9], 0.7232142857142857, Ops::mulc(Lam[5], 1.1571428571428573)));
    K[185] = Ops::fmac(w42, -0.14464285714285716, Ops::mulc(w15, -0.2892857142857143));
    K[186] = Ops::fmac(w49, 1.4464285714285714, Ops::mulc(w39, 0.5785714285714286));
    K[187] = Ops::fmac(w25, -0.14464285714285716, Ops::fmac(w15, 0.7232142857142857, Ops::mulc(w11, 0.5785714285714286)));
    K[188] = Ops::fmac(w57, 1.4464285714285714, Ops::mulc(w36, 0.5785714285714286));
    K[189] = Ops::fmac(w6, 1.1571428571428573, Ops::mulc(Lam[7], 1.4464285714285714));
    K[190] = Ops::fmac(Lam[9], -0.43392857142857144, Ops::fmac(Lam[8], 0.2892857142857143, Ops::mulc(Lam[7], -0.43392857142857144)));
    K[191] = Ops::fmac(w26, -0.14464285714285716, Ops::fmac(w9, 0.7232142857142857, Ops::mulc(w1, 0.5785714285714286)));
    K[192] = Ops::fmac(w29, -0.14464285714285716, Ops::mulc(w9, -0.2892857142857143));
    K[193] = Ops::fmac(w48, 1.4464285714285714, Ops::mulc(w35, 0.5785714285714286));
    K[194] = Ops::fmac(w52, 1.4464285714285714, Ops::mulc(w40, 0.5785714285714286));
    K[195] = Ops::fmac(w26, 1.1571428571428573, Ops::mulc(Lam[9], 1.4464285714285714));
    K[196] = Ops::fmac(w31, -0.14464285714285716, Ops::mulc(w1, -0.2892857142857143));
    K[197] = Ops::fmac(w9, 0.5785714285714286, Ops::fmac(w6, -0.14464285714285716, Ops::mulc(w1, 0.7232142857142857)));
    K[198] = Ops::fmac(w49, 1.4464285714285714, Ops::mulc(w41, 0.5785714285714286));
    K[199] = Ops::fmac(w54, 1.4464285714285714, Ops::mulc(w19, 0.5785714285714286));
    K[200] = Ops::fmac(w59, 3.4714285714285715, Ops::mulc(Lam[7], 3.4714285714285715));
    K[201] = Ops::fmac(w59, 1.7357142857142858, Ops::fmac(w1, 1.7357142857142858, Ops::mulc(Lam[8], 3.4714285714285715)));
    K[202] = Ops::fmac(w55, 3.4714285714285715, Ops::mulc(w27, 1.7357142857142858));
    K[203] = Ops::fmac(w60, 1.7357142857142858, Ops::fmac(w0, 1.7357142857142858, Ops::mulc(Lam[3], 3.4714285714285715)));
    K[204] = Ops::fmac(w58, 3.4714285714285715, Ops::mulc(Lam[0], 3.4714285714285715));
    K[205] = Ops::fmac(w53, 3.4714285714285715, Ops::mulc(w29, 1.7357142857142858));
    K[206] = Ops::fmac(w58, 1.7357142857142858, Ops::fmac(w2, 1.7357142857142858, Ops::mulc(Lam[2], 3.4714285714285715)));
    K[207] = Ops::fmac(w6, 3.4714285714285715, Ops::fmac(w5, 3.4714285714285715, Ops::mulc(w3, 3.4714285714285715)));
    K[208] = Ops::fmac(w47, 3.4714285714285715, Ops::mulc(w31, 1.7357142857142858));
    K[209] = Ops::fmac(w60, 3.4714285714285715, Ops::mulc(Lam[9], 3.4714285714285715));
  }
  template <class Ops> __device__ __forceinline__ static void helmholtz_upper(const typename Ops::T* Lam, const typename Ops::T& vol, typename Ops::T* K) {
    const typename Ops::T w0 = Ops::add(Lam[1], Lam[2]);
    const typename Ops::T w1 = Ops::add(Lam[3], Lam[6]);
    const typename Ops::T w2 = Ops::add(Lam[5], Lam[8]);
    const typename Ops::T w3 = Ops::add(Lam[0], Lam[3]);
    const typename Ops::T w4 = Ops::add(Lam[1], Lam[4]);
    const typename Ops::T w5 = Ops::add(Lam[2], Lam[7]);
    const typename Ops::T w6 = Ops::add(Lam[8], Lam[9]);
    const typename Ops::T w7 = Ops::add(Lam[5], Lam[6]);
    const typename Ops::T w8 = Ops::add(Lam[1], Lam[3]);
    const typename Ops::T w9 = Ops::add(Lam[2], Lam[5]);
    const typename Ops::T w10 = Ops::add(Lam[6], Lam[8]);
    const typename Ops::T w11 = Ops::add(Lam[1], Lam[5]);
    const typename Ops::T w12 = Ops::add(Lam[1], Lam[6]);
    const typename Ops::T w13 = Ops::add(Lam[2], Lam[3]);
    const typename Ops::T w14 = Ops::add(Lam[2], Lam[8]);
    const typename Ops::T w15 = Ops::add(Lam[3], Lam[8]);
    const typename Ops::T w16 = Ops::add(Lam[0], w0);
    const typename Ops::T w17 = Ops::add(Lam[4], Lam[5]);
    const typename Ops::T w18 = Ops::add(Lam[4], Lam[6]);
    const typename Ops::T w19 = Ops::add(Lam[7], w2);
    const typename Ops::T w20 = Ops::add(Lam[9], w1);
    const typename Ops::T w21 = Ops::add(Lam[0], Lam[1]);
    const typename Ops::T w22 = Ops::add(Lam[0], Lam[2]);
    const typename Ops::T w23 = Ops::add(Lam[3], Lam[9]);
    const typename Ops::T w24 = Ops::add(Lam[5], Lam[7]);
    const typename Ops::T w25 = Ops::add(Lam[6], Lam[9]);
    const typename Ops::T w26 = Ops::add(Lam[7], Lam[8]);
    const typename Ops::T w27 = Ops::add(w0, w3);
    const typename Ops::T w28 = Ops::add(w0, w10);
    const typename Ops::T w29 = Ops::add(w1, w6);
    const typename Ops::T w30 = Ops::add(w1, w9);
    const typename Ops::T w31 = Ops::add(w2, w5);
    const typename Ops::T w32 = Ops::add(w2, w8);
    const typename Ops::T w33 = Ops::add(Lam[1], w3);
    const typename Ops::T w34 = Ops::add(Lam[2], w3);
    const typename Ops::T w35 = Ops::add(Lam[3], w6);
    const typename Ops::T w36 = Ops::add(Lam[4], w7);
    const typename Ops::T w37 = Ops::add(Lam[5], w4);
    const typename Ops::T w38 = Ops::add(Lam[5], w5);
    const typename Ops::T w39 = Ops::add(Lam[6], w4);
    const typename Ops::T w40 = Ops::add(Lam[6], w6);
    const typename Ops::T w41 = Ops::add(Lam[8], w5);
    const typename Ops::T w42 = Ops::add(w4, w7);
    const typename Ops::T w43 = Ops::fmac(Lam[1], -5.0, Lam[0]);
    const typename Ops::T w44 = Ops::fmac(Lam[2], -5.0, Lam[0]);
    const typename Ops::T w45 = Ops::fmac(Lam[3], -5.0, Lam[0]);
    const typename Ops::T w46 = Ops::fmac(Lam[4], -0.2, Lam[1]);
    const typename Ops::T w47 = Ops::fmac(w20, 0.5, Lam[1]);
    const typename Ops::T w48 = Ops::fmac(Lam[7], -0.2, Lam[2]);
    const typename Ops::T w49 = Ops::fmac(Lam[9], -0.2, Lam[3]);
    const typename Ops::T w50 = Ops::fmac(Lam[5], -5.0, Lam[4]);
    const typename Ops::T w51 = Ops::fmac(Lam[6], -5.0, Lam[4]);
    const typename Ops::T w52 = Ops::fmac(Lam[7], -0.2, Lam[5]);
    const typename Ops::T w53 = Ops::fmac(w16, 0.5, Lam[5]);
    const typename Ops::T w54 = Ops::fmac(Lam[9], -0.2, Lam[6]);
    const typename Ops::T w55 = Ops::fmac(w19, 0.5, Lam[6]);
    const typename Ops::T w56 = Ops::fmac(Lam[8], -5.0, Lam[7]);
    const typename Ops::T w57 = Ops::fmac(Lam[9], -0.2, Lam[8]);
    const typename Ops::T w58 = Ops::add(w4, w20);
    const typename Ops::T w59 = Ops::add(w16, w17);
    const typename Ops::T w60 = Ops::add(w18, w19);
    const typename Ops::T m0 = Ops::mulc(vol, 0.0035714285714285713);
    const typename Ops::T m1 = Ops::mulc(vol, 0.0004464285714285714);
    const typename Ops::T m2 = Ops::mulc(vol, -0.0026785714285714286);
    const typename Ops::T m3 = Ops::mulc(vol, 0.0013392857142857143);
    const typename Ops::T m4 = Ops::mulc(vol, 0.0006696428571428571);
    const typename Ops::T m5 = Ops::mulc(vol, 0.0040178571428571425);
    const typename Ops::T m6 = Ops::mulc(vol, 0.008035714285714285);
    const typename Ops::T m7 = Ops::mulc(vol, 0.024107142857142858);
    const typename Ops::T m8 = Ops::mulc(vol, -0.012053571428571429);
    const typename Ops::T m9 = Ops::mulc(vol, 0.012053571428571429);
    const typename Ops::T m10 = Ops::mulc(vol, -0.0060267857142857146);
    const typename Ops::T m11 = Ops::mulc(vol, 0.09642857142857143);
    const typename Ops::T m12 = Ops::mulc(vol, 0.048214285714285716);
    K[0] = Ops::fmac(Lam[0], 0.35714285714285715, m0);
    K[1] = Ops::fmac(Lam[1], 0.06785714285714285, m1);
    K[2] = Ops::fmac(Lam[2], 0.06785714285714285, m1);
    K[3] = Ops::fmac(Lam[3], 0.06785714285714285, m1);
    K[4] = Ops::fmac(Lam[1], 0.36964285714285716, Ops::fmac(Lam[0], -0.20892857142857144, m2));
    K[5] = Ops::fmac(Lam[1], -0.20892857142857144, Ops::fmac(Lam[0], 0.08035714285714286, m3));
    K[6] = Ops::fmac(Lam[2], 0.36964285714285716, Ops::fmac(Lam[0], -0.20892857142857144, m2));
    K[7] = Ops::fmac(Lam[2], -0.20892857142857144, Ops::fmac(Lam[0], 0.08035714285714286, m3));
    K[8] = Ops::fmac(Lam[3], 0.36964285714285716, Ops::fmac(Lam[0], -0.20892857142857144, m2));
    K[9] = Ops::fmac(Lam[3], -0.20892857142857144, Ops::fmac(Lam[0], 0.08035714285714286, m3));
    K[10] = Ops::fmac(w0, 0.08035714285714286, m4);
    K[11] = Ops::fmac(w0, 0.08035714285714286, m4);
    K[12] = Ops::fmac(w8, 0.08035714285714286, m4);
    K[13] = Ops::fmac(w8, 0.08035714285714286, m4);
    K[14] = Ops::fmac(w13, 0.08035714285714286, m4);
    K[15] = Ops::fmac(w13, 0.08035714285714286, m4);
    K[16] = Ops::fmac(w0, -0.09642857142857143, Ops::fmac(Lam[0], 0.19285714285714287, m5));
    K[17] = Ops::fmac(w8, -0.09642857142857143, Ops::fmac(Lam[0], 0.19285714285714287, m5));
    K[18] = Ops::fmac(w13, -0.09642857142857143, Ops::fmac(Lam[0], 0.19285714285714287, m5));
    K[19] = Ops::fmac(w0, 0.19285714285714287, Ops::fmac(Lam[3], 0.19285714285714287, m6));
    K[20] = Ops::fmac(Lam[4], 0.35714285714285715, m0);
    K[21] = Ops::fmac(Lam[5], 0.06785714285714285, m1);
    K[22] = Ops::fmac(Lam[6], 0.06785714285714285, m1);
    K[23] = Ops::fmac(Lam[4], 0.08035714285714286, Ops::fmac(Lam[1], -0.20892857142857144, m3));
    K[24] = Ops::fmac(Lam[4], -0.20892857142857144, Ops::fmac(Lam[1], 0.36964285714285716, m2));
    K[25] = Ops::fmac(w11, 0.08035714285714286, m4);
    K[26] = Ops::fmac(w11, 0.08035714285714286, m4);
    K[27] = Ops::fmac(w12, 0.08035714285714286, m4);
    K[28] = Ops::fmac(w12, 0.08035714285714286, m4);
    K[29] = Ops::fmac(Lam[5], 0.36964285714285716, Ops::fmac(Lam[4], -0.20892857142857144, m2));
    K[30] = Ops::fmac(Lam[5], -0.20892857142857144, Ops::fmac(Lam[4], 0.08035714285714286, m3));
    K[31] = Ops::fmac(Lam[6], 0.36964285714285716, Ops::fmac(Lam[4], -0.20892857142857144, m2));
    K[32] = Ops::fmac(Lam[6], -0.20892857142857144, Ops::fmac(Lam[4], 0.08035714285714286, m3));
    K[33] = Ops::fmac(w7, 0.08035714285714286, m4);
    K[34] = Ops::fmac(w7, 0.08035714285714286, m4);
    K[35] = Ops::fmac(w11, -0.09642857142857143, Ops::fmac(Lam[4], 0.19285714285714287, m5));
    K[36] = Ops::fmac(w12, -0.09642857142857143, Ops::fmac(Lam[4], 0.19285714285714287, m5));
    K[37] = Ops::fmac(w7, 0.19285714285714287, Ops::fmac(Lam[1], 0.19285714285714287, m6));
    K[38] = Ops::fmac(w7, -0.09642857142857143, Ops::fmac(Lam[4], 0.19285714285714287, m5));
    K[39] = Ops::fmac(Lam[7], 0.35714285714285715, m0);
    K[40] = Ops::fmac(Lam[8], 0.06785714285714285, m1);
    K[41] = Ops::fmac(w9, 0.08035714285714286, m4);
    K[42] = Ops::fmac(w9, 0.08035714285714286, m4);
    K[43] = Ops::fmac(Lam[7], 0.08035714285714286, Ops::fmac(Lam[2], -0.20892857142857144, m3));
    K[44] = Ops::fmac(Lam[7], -0.20892857142857144, Ops::fmac(Lam[2], 0.36964285714285716, m2));
    K[45] = Ops::fmac(w14, 0.08035714285714286, m4);
    K[46] = Ops::fmac(w14, 0.08035714285714286, m4);
    K[47] = Ops::fmac(Lam[7], 0.08035714285714286, Ops::fmac(Lam[5], -0.20892857142857144, m3));
    K[48] = Ops::fmac(Lam[7], -0.20892857142857144, Ops::fmac(Lam[5], 0.36964285714285716, m2));
    K[49] = Ops::fmac(w2, 0.08035714285714286, m4);
    K[50] = Ops::fmac(w2, 0.08035714285714286, m4);
    K[51] = Ops::fmac(Lam[8], 0.36964285714285716, Ops::fmac(Lam[7], -0.20892857142857144, m2));
    K[52] = Ops::fmac(Lam[8], -0.20892857142857144, Ops::fmac(Lam[7], 0.08035714285714286, m3));
    K[53] = Ops::fmac(w9, -0.09642857142857143, Ops::fmac(Lam[7], 0.19285714285714287, m5));
    K[54] = Ops::fmac(w2, 0.19285714285714287, Ops::fmac(Lam[2], 0.19285714285714287, m6));
    K[55] = Ops::fmac(w14, -0.09642857142857143, Ops::fmac(Lam[7], 0.19285714285714287, m5));
    K[56] = Ops::fmac(w2, -0.09642857142857143, Ops::fmac(Lam[7], 0.19285714285714287, m5));
    K[57] = Ops::fmac(Lam[9], 0.35714285714285715, m0);
    K[58] = Ops::fmac(w1, 0.08035714285714286, m4);
    K[59] = Ops::fmac(w1, 0.08035714285714286, m4);
    K[60] = Ops::fmac(w15, 0.08035714285714286, m4);
    K[61] = Ops::fmac(w15, 0.08035714285714286, m4);
    K[62] = Ops::fmac(Lam[9], 0.08035714285714286, Ops::fmac(Lam[3], -0.20892857142857144, m3));
    K[63] = Ops::fmac(Lam[9], -0.20892857142857144, Ops::fmac(Lam[3], 0.36964285714285716, m2));
    K[64] = Ops::fmac(w10, 0.08035714285714286, m4);
    K[65] = Ops::fmac(w10, 0.08035714285714286, m4);
    K[66] = Ops::fmac(Lam[9], 0.08035714285714286, Ops::fmac(Lam[6], -0.20892857142857144, m3));
    K[67] = Ops::fmac(Lam[9], -0.20892857142857144, Ops::fmac(Lam[6], 0.36964285714285716, m2));
    K[68] = Ops::fmac(Lam[9], 0.08035714285714286, Ops::fmac(Lam[8], -0.20892857142857144, m3));
    K[69] = Ops::fmac(Lam[9], -0.20892857142857144, Ops::fmac(Lam[8], 0.36964285714285716, m2));
    K[70] = Ops::fmac(w1, 0.19285714285714287, Ops::fmac(Lam[8], 0.19285714285714287, m6));
    K[71] = Ops::fmac(w1, -0.09642857142857143, Ops::fmac(Lam[9], 0.19285714285714287, m5));
    K[72] = Ops::fmac(w15, -0.09642857142857143, Ops::fmac(Lam[9], 0.19285714285714287, m5));
    K[73] = Ops::fmac(w10, -0.09642857142857143, Ops::fmac(Lam[9], 0.19285714285714287, m5));
    K[74] = Ops::fmac(w4, 1.1571428571428573, Ops::fmac(Lam[0], 1.4464285714285714, m7));
    K[75] = Ops::fmac(Lam[4], -0.43392857142857144, Ops::fmac(Lam[1], 0.2892857142857143, Ops::fmac(Lam[0], -0.43392857142857144, m8)));
    K[76] = Ops::fmac(w0, 0.5785714285714286, Ops::fmac(Lam[5], 1.1571428571428573, Ops::fmac(Lam[0], 0.7232142857142857, m9)));
    K[77] = Ops::fmac(w21, -0.14464285714285716, Ops::fmac(Lam[5], -0.43392857142857144, Ops::fmac(Lam[2], -0.2892857142857143, m10)));
    K[78] = Ops::fmac(w8, 0.5785714285714286, Ops::fmac(Lam[6], 1.1571428571428573, Ops::fmac(Lam[0], 0.7232142857142857, m9)));
    K[79] = Ops::fmac(w21, -0.14464285714285716, Ops::fmac(Lam[6], -0.43392857142857144, Ops::fmac(Lam[3], -0.2892857142857143, m10)));
    K[80] = Ops::fmac(w17, -0.14464285714285716, Ops::fmac(Lam[2], -0.43392857142857144, Ops::fmac(Lam[1], -0.2892857142857143, m10)));
    K[81] = Ops::fmac(w37, -0.14464285714285716, Ops::mulc(Lam[2], -0.2892857142857143));
    K[82] = Ops::fmac(w18, -0.14464285714285716, Ops::fmac(Lam[3], -0.43392857142857144, Ops::fmac(Lam[1], -0.2892857142857143, m10)));
    K[83] = Ops::fmac(w39, -0.14464285714285716, Ops::mulc(Lam[3], -0.2892857142857143));
    K[84] = Ops::mulc(w30, -0.14464285714285716);
    K[85] = Ops::mulc(w30, -0.14464285714285716);
    K[86] = Ops::fmac(w44, -0.2892857142857143, Ops::mulc(w37, 0.5785714285714286));
    K[87] = Ops::fmac(w45, -0.2892857142857143, Ops::mulc(w39, 0.5785714285714286));
    K[88] = Ops::fmac(w21, -0.14464285714285716, Ops::fmac(w13, 0.7232142857142857, Ops::mulc(w7, 0.5785714285714286)));
    K[89] = Ops::fmac(w42, -0.14464285714285716, Ops::fmac(w13, -0.2892857142857143, m8));
    K[90] = Ops::fmac(w21, 1.1571428571428573, Ops::fmac(Lam[4], 1.4464285714285714, m7));
    K[91] = Ops::fmac(w22, -0.14464285714285716, Ops::fmac(Lam[5], -0.43392857142857144, Ops::fmac(Lam[1], -0.2892857142857143, m10)));
    K[92] = Ops::mulc(w53, -0.2892857142857143);
    K[93] = Ops::fmac(w3, -0.14464285714285716, Ops::fmac(Lam[6], -0.43392857142857144, Ops::fmac(Lam[1], -0.2892857142857143, m10)));
    K[94] = Ops::fmac(w33, -0.14464285714285716, Ops::mulc(Lam[6], -0.2892857142857143));
    K[95] = Ops::fmac(w11, 0.5785714285714286, Ops::fmac(Lam[4], 0.7232142857142857, Ops::fmac(Lam[2], 1.1571428571428573, m9)));
    K[96] = Ops::fmac(w4, -0.14464285714285716, Ops::fmac(Lam[5], -0.2892857142857143, Ops::fmac(Lam[2], -0.43392857142857144, m10)));
    K[97] = Ops::fmac(w12, 0.5785714285714286, Ops::fmac(Lam[4], 0.7232142857142857, Ops::fmac(Lam[3], 1.1571428571428573, m9)));
    K[98] = Ops::fmac(w4, -0.14464285714285716, Ops::fmac(Lam[6], -0.2892857142857143, Ops::fmac(Lam[3], -0.43392857142857144, m10)));
    K[99] = Ops::mulc(w30, -0.14464285714285716);
    K[100] = Ops::mulc(w30, -0.14464285714285716);
    K[101] = Ops::fmac(w50, -0.2892857142857143, Ops::mulc(w16, 0.5785714285714286));
    K[102] = Ops::fmac(w51, -0.2892857142857143, Ops::mulc(w33, 0.5785714285714286));
    K[103] = Ops::fmac(w27, -0.14464285714285716, Ops::fmac(w7, -0.2892857142857143, m8));
    K[104] = Ops::fmac(w13, 0.5785714285714286, Ops::fmac(w7, 0.7232142857142857, Ops::mulc(w4, -0.14464285714285716)));
    K[105] = Ops::fmac(w5, 1.1571428571428573, Ops::fmac(Lam[0], 1.4464285714285714, m7));
    K[106] = Ops::fmac(Lam[7], -0.43392857142857144, Ops::fmac(Lam[2], 0.2892857142857143, Ops::fmac(Lam[0], -0.43392857142857144, m8)));
    K[107] = Ops::fmac(w13, 0.5785714285714286, Ops::fmac(Lam[8], 1.1571428571428573, Ops::fmac(Lam[0], 0.7232142857142857, m9)));
    K[108] = Ops::fmac(w22, -0.14464285714285716, Ops::fmac(Lam[8], -0.43392857142857144, Ops::fmac(Lam[3], -0.2892857142857143, m10)));
    K[109] = Ops::fmac(w38, -0.14464285714285716, Ops::mulc(Lam[1], -0.2892857142857143));
    K[110] = Ops::fmac(w24, -0.14464285714285716, Ops::fmac(Lam[2], -0.2892857142857143, Ops::fmac(Lam[1], -0.43392857142857144, m10)));
    K[111] = Ops::mulc(w32, -0.14464285714285716);
    K[112] = Ops::mulc(w32, -0.14464285714285716);
    K[113] = Ops::fmac(w26, -0.14464285714285716, Ops::fmac(Lam[3], -0.43392857142857144, Ops::fmac(Lam[2], -0.2892857142857143, m10)));
    K[114] = Ops::fmac(w41, -0.14464285714285716, Ops::mulc(Lam[3], -0.2892857142857143));
    K[115] = Ops::fmac(w43, -0.2892857142857143, Ops::mulc(w38, 0.5785714285714286));
    K[116] = Ops::fmac(w22, -0.14464285714285716, Ops::fmac(w8, 0.7232142857142857, Ops::mulc(w2, 0.5785714285714286)));
    K[117] = Ops::fmac(w45, -0.2892857142857143, Ops::mulc(w41, 0.5785714285714286));
    K[118] = Ops::fmac(w31, -0.14464285714285716, Ops::fmac(w8, -0.2892857142857143, m8));
    K[119] = Ops::fmac(w22, 1.1571428571428573, Ops::fmac(Lam[7], 1.4464285714285714, m7));
    K[120] = Ops::fmac(w3, -0.14464285714285716, Ops::fmac(Lam[8], -0.43392857142857144, Ops::fmac(Lam[2], -0.2892857142857143, m10)));
    K[121] = Ops::fmac(w34, -0.14464285714285716, Ops::mulc(Lam[8], -0.2892857142857143));
    K[122] = Ops::fmac(w5, -0.14464285714285716, Ops::fmac(Lam[5], -0.2892857142857143, Ops::fmac(Lam[1], -0.43392857142857144, m10)));
    K[123] = Ops::fmac(w9, 0.5785714285714286, Ops::fmac(Lam[7], 0.7232142857142857, Ops::fmac(Lam[1], 1.1571428571428573, m9)));
    K[124] = Ops::mulc(w32, -0.14464285714285716);
    K[125] = Ops::mulc(w32, -0.14464285714285716);
    K[126] = Ops::fmac(w14, 0.5785714285714286, Ops::fmac(Lam[7], 0.7232142857142857, Ops::fmac(Lam[3], 1.1571428571428573, m9)));
    K[127] = Ops::fmac(w5, -0.14464285714285716, Ops::fmac(Lam[8], -0.2892857142857143, Ops::fmac(Lam[3], -0.43392857142857144, m10)));
    K[128] = Ops::fmac(w52, 1.4464285714285714, Ops::mulc(w16, 0.5785714285714286));
    K[129] = Ops::fmac(w27, -0.14464285714285716, Ops::fmac(w2, -0.2892857142857143, m8));
    K[130] = Ops::fmac(w56, -0.2892857142857143, Ops::mulc(w34, 0.5785714285714286));
    K[131] = Ops::fmac(w8, 0.5785714285714286, Ops::fmac(w5, -0.14464285714285716, Ops::mulc(w2, 0.7232142857142857)));
    K[132] = Ops::fmac(w23, 1.1571428571428573, Ops::fmac(Lam[0], 1.4464285714285714, m7));
    K[133] = Ops::fmac(Lam[9], -0.43392857142857144, Ops::fmac(Lam[3], 0.2892857142857143, Ops::fmac(Lam[0], -0.43392857142857144, m8)));
    K[134] = Ops::mulc(w28, -0.14464285714285716);
    K[135] = Ops::mulc(w28, -0.14464285714285716);
    K[136] = Ops::mulc(w47, -0.2892857142857143);
    K[137] = Ops::fmac(w25, -0.14464285714285716, Ops::fmac(Lam[3], -0.2892857142857143, Ops::fmac(Lam[1], -0.43392857142857144, m10)));
    K[138] = Ops::fmac(w35, -0.14464285714285716, Ops::mulc(Lam[2], -0.2892857142857143));
    K[139] = Ops::fmac(w6, -0.14464285714285716, Ops::fmac(Lam[3], -0.2892857142857143, Ops::fmac(Lam[2], -0.43392857142857144, m10)));
    K[140] = Ops::fmac(w10, 0.5785714285714286, Ops::fmac(w3, -0.14464285714285716, Ops::mulc(w0, 0.7232142857142857)));
    K[141] = Ops::fmac(w43, -0.2892857142857143, Ops::mulc(w20, 0.5785714285714286));
    K[142] = Ops::fmac(w44, -0.2892857142857143, Ops::mulc(w35, 0.5785714285714286));
    K[143] = Ops::fmac(w29, -0.14464285714285716, Ops::fmac(w0, -0.2892857142857143, m8));
    K[144] = Ops::fmac(w3, 1.1571428571428573, Ops::fmac(Lam[9], 1.4464285714285714, m7));
    K[145] = Ops::mulc(w28, -0.14464285714285716);
    K[146] = Ops::mulc(w28, -0.14464285714285716);
    K[147] = Ops::fmac(w23, -0.14464285714285716, Ops::fmac(Lam[6], -0.2892857142857143, Ops::fmac(Lam[1], -0.43392857142857144, m10)));
    K[148] = Ops::fmac(w1, 0.5785714285714286, Ops::fmac(Lam[9], 0.7232142857142857, Ops::fmac(Lam[1], 1.1571428571428573, m9)));
    K[149] = Ops::fmac(w23, -0.14464285714285716, Ops::fmac(Lam[8], -0.2892857142857143, Ops::fmac(Lam[2], -0.43392857142857144, m10)));
    K[150] = Ops::fmac(w15, 0.5785714285714286, Ops::fmac(Lam[9], 0.7232142857142857, Ops::fmac(Lam[2], 1.1571428571428573, m9)));
    K[151] = Ops::fmac(w27, -0.14464285714285716, Ops::fmac(w10, -0.2892857142857143, m8));
    K[152] = Ops::fmac(w54, 1.4464285714285714, Ops::mulc(w33, 0.5785714285714286));
    K[153] = Ops::fmac(w57, 1.4464285714285714, Ops::mulc(w34, 0.5785714285714286));
    K[154] = Ops::fmac(w23, -0.14464285714285716, Ops::fmac(w10, 0.7232142857142857, Ops::mulc(w0, 0.5785714285714286)));
    K[155] = Ops::fmac(w24, 1.1571428571428573, Ops::fmac(Lam[4], 1.4464285714285714, m7));
    K[156] = Ops::fmac(Lam[7], -0.43392857142857144, Ops::fmac(Lam[5], 0.2892857142857143, Ops::fmac(Lam[4], -0.43392857142857144, m8)));
    K[157] = Ops::fmac(w7, 0.5785714285714286, Ops::fmac(Lam[8], 1.1571428571428573, Ops::fmac(Lam[4], 0.7232142857142857, m9)));
    K[158] = Ops::fmac(w17, -0.14464285714285716, Ops::fmac(Lam[8], -0.43392857142857144, Ops::fmac(Lam[6], -0.2892857142857143, m10)));
    K[159] = Ops::fmac(w26, -0.14464285714285716, Ops::fmac(Lam[6], -0.43392857142857144, Ops::fmac(Lam[5], -0.2892857142857143, m10)));
    K[160] = Ops::mulc(w55, -0.2892857142857143);
    K[161] = Ops::fmac(w46, 1.4464285714285714, Ops::mulc(w38, 0.5785714285714286));
    K[162] = Ops::fmac(w17, -0.14464285714285716, Ops::fmac(w14, 0.5785714285714286, Ops::mulc(w12, 0.7232142857142857)));
    K[163] = Ops::fmac(w31, -0.14464285714285716, Ops::fmac(w12, -0.2892857142857143, m8));
    K[164] = Ops::fmac(w51, -0.2892857142857143, Ops::mulc(w19, 0.5785714285714286));
    K[165] = Ops::fmac(w17, 1.1571428571428573, Ops::fmac(Lam[7], 1.4464285714285714, m7));
    K[166] = Ops::fmac(w18, -0.14464285714285716, Ops::fmac(Lam[8], -0.43392857142857144, Ops::fmac(Lam[5], -0.2892857142857143, m10)));
    K[167] = Ops::fmac(w36, -0.14464285714285716, Ops::mulc(Lam[8], -0.2892857142857143));
    K[168] = Ops::fmac(w2, 0.5785714285714286, Ops::fmac(Lam[7], 0.7232142857142857, Ops::fmac(Lam[6], 1.1571428571428573, m9)));
    K[169] = Ops::fmac(w24, -0.14464285714285716, Ops::fmac(Lam[8], -0.2892857142857143, Ops::fmac(Lam[6], -0.43392857142857144, m10)));
    K[170] = Ops::fmac(w48, 1.4464285714285714, Ops::mulc(w37, 0.5785714285714286));
    K[171] = Ops::fmac(w42, -0.14464285714285716, Ops::fmac(w14, -0.2892857142857143, m8));
    K[172] = Ops::fmac(w24, -0.14464285714285716, Ops::fmac(w14, 0.7232142857142857, Ops::mulc(w12, 0.5785714285714286)));
    K[173] = Ops::fmac(w56, -0.2892857142857143, Ops::mulc(w36, 0.5785714285714286));
    K[174] = Ops::fmac(w25, 1.1571428571428573, Ops::fmac(Lam[4], 1.4464285714285714, m7));
    K[175] = Ops::fmac(Lam[9], -0.43392857142857144, Ops::fmac(Lam[6], 0.2892857142857143, Ops::fmac(Lam[4], -0.43392857142857144, m8)));
    K[176] = Ops::fmac(w40, -0.14464285714285716, Ops::mulc(Lam[5], -0.2892857142857143));
    K[177] = Ops::fmac(w6, -0.14464285714285716, Ops::fmac(Lam[6], -0.2892857142857143, Ops::fmac(Lam[5], -0.43392857142857144, m10)));
    K[178] = Ops::fmac(w18, -0.14464285714285716, Ops::fmac(w15, 0.5785714285714286, Ops::mulc(w11, 0.7232142857142857)));
    K[179] = Ops::fmac(w46, 1.4464285714285714, Ops::mulc(w20, 0.5785714285714286));
    K[180] = Ops::fmac(w29, -0.14464285714285716, Ops::fmac(w11, -0.2892857142857143, m8));
    K[181] = Ops::fmac(w50, -0.2892857142857143, Ops::mulc(w40, 0.5785714285714286));
    K[182] = Ops::fmac(w18, 1.1571428571428573, Ops::fmac(Lam[9], 1.4464285714285714, m7));
    K[183] = Ops::fmac(w25, -0.14464285714285716, Ops::fmac(Lam[8], -0.2892857142857143, Ops::fmac(Lam[5], -0.43392857142857144, m10)));
    K[184] = Ops::fmac(w10, 0.5785714285714286, Ops::fmac(Lam[9], 0.7232142857142857, Ops::fmac(Lam[5], 1.1571428571428573, m9)));
    K[185] = Ops::fmac(w42, -0.14464285714285716, Ops::fmac(w15, -0.2892857142857143, m8));
    K[186] = Ops::fmac(w49, 1.4464285714285714, Ops::mulc(w39, 0.5785714285714286));
    K[187] = Ops::fmac(w25, -0.14464285714285716, Ops::fmac(w15, 0.7232142857142857, Ops::mulc(w11, 0.5785714285714286)));
    K[188] = Ops::fmac(w57, 1.4464285714285714, Ops::mulc(w36, 0.5785714285714286));
    K[189] = Ops::fmac(w6, 1.1571428571428573, Ops::fmac(Lam[7], 1.4464285714285714, m7));
    K[190] = Ops::fmac(Lam[9], -0.43392857142857144, Ops::fmac(Lam[8], 0.2892857142857143, Ops::fmac(Lam[7], -0.43392857142857144, m8)));
    K[191] = Ops::fmac(w26, -0.14464285714285716, Ops::fmac(w9, 0.7232142857142857, Ops::mulc(w1, 0.5785714285714286)));
    K[192] = Ops::fmac(w29, -0.14464285714285716, Ops::fmac(w9, -0.2892857142857143, m8));
    K[193] = Ops::fmac(w48, 1.4464285714285714, Ops::mulc(w35, 0.5785714285714286));
    K[194] = Ops::fmac(w52, 1.4464285714285714, Ops::mulc(w40, 0.5785714285714286));
    K[195] = Ops::fmac(w26, 1.1571428571428573, Ops::fmac(Lam[9], 1.4464285714285714, m7));
    K[196] = Ops::fmac(w31, -0.14464285714285716, Ops::fmac(w1, -0.2892857142857143, m8));
    K[197] = Ops::fmac(w9, 0.5785714285714286, Ops::fmac(w6, -0.14464285714285716, Ops::mulc(w1, 0.7232142857142857)));
    K[198] = Ops::fmac(w49, 1.4464285714285714, Ops::mulc(w41, 0.5785714285714286));
    K[199] = Ops::fmac(w54, 1.4464285714285714, Ops::mulc(w19, 0.5785714285714286));
    K[200] = Ops::fmac(w59, 3.4714285714285715, Ops::fmac(Lam[7], 3.4714285714285715, m11));
    K[201] = Ops::fmac(w59, 1.7357142857142858, Ops::fmac(w1, 1.7357142857142858, Ops::fmac(Lam[8], 3.4714285714285715, m12)));
    K[202] = Ops::fmac(w55, 3.4714285714285715, Ops::fmac(w27, 1.7357142857142858, m12));
    K[203] = Ops::fmac(w60, 1.7357142857142858, Ops::fmac(w0, 1.7357142857142858, Ops::fmac(Lam[3], 3.4714285714285715, m12)));
    K[204] = Ops::fmac(w58, 3.4714285714285715, Ops::fmac(Lam[0], 3.4714285714285715, m11));
    K[205] = Ops::fmac(w53, 3.4714285714285715, Ops::fmac(w29, 1.7357142857142858, m12));
    K[206] = Ops::fmac(w58, 1.7357142857142858, Ops::fmac(w2, 1.7357142857142858, Ops::fmac(Lam[2], 3.4714285714285715, m12)));
    K[207] = Ops::fmac(w6, 3.4714285714285715, Ops::fmac(w5, 3.4714285714285715, Ops::fmac(w3, 3.4714285714285715, m11)));
    K[208] = Ops::fmac(w47, 3.4714285714285715, Ops::fmac(w31, 1.7357142857142858, m12));
    K[209] = Ops::fmac(w60, 3.4714285714285715, Ops::fmac(Lam[9], 3.4714285714285715, m11));
  }
  template <class Ops> __device__ __forceinline__ static void mass_upper(const typename Ops::T& vol, typename Ops::T* K) {
    const typename Ops::T m0 = Ops::mulc(vol, 0.0035714285714285713);
    const typename Ops::T m1 = Ops::mulc(vol, 0.0004464285714285714);
    const typename Ops::T m2 = Ops::mulc(vol, -0.0026785714285714286);
    const typename Ops::T m3 = Ops::mulc(vol, 0.0013392857142857143);
    const typename Ops::T m4 = Ops::mulc(vol, 0.0006696428571428571);
    const typename Ops::T m5 = Ops::mulc(vol, 0.0040178571428571425);
    const typename Ops::T m6 = Ops::mulc(vol, 0.008035714285714285);
    const typename Ops::T m7 = Ops::mulc(vol, 0.024107142857142858);
    const typename Ops::T m8 = Ops::mulc(vol, -0.012053571428571429);
    const typename Ops::T m9 = Ops::mulc(vol, 0.012053571428571429);
    const typename Ops::T m10 = Ops::mulc(vol, -0.0060267857142857146);
    const typename Ops::T m11 = Ops::mulc(vol, 0.09642857142857143);
    const typename Ops::T m12 = Ops::mulc(vol, 0.048214285714285716);
    K[0] = m0;
    K[1] = m1;
    K[2] = m1;
    K[3] = m1;
    K[4] = m2;
    K[5] = m3;
    K[6] = m2;
    K[7] = m3;
    K[8] = m2;
    K[9] = m3;
    K[10] = m4;
    K[11] = m4;
    K[12] = m4;
    K[13] = m4;
    K[14] = m4;
    K[15] = m4;
    K[16] = m5;
    K[17] = m5;
    K[18] = m5;
    K[19] = m6;
    K[20] = m0;
    K[21] = m1;
    K[22] = m1;
    K[23] = m3;
    K[24] = m2;
    K[25] = m4;
    K[26] = m4;
    K[27] = m4;
    K[28] = m4;
    K[29] = m2;
    K[30] = m3;
    K[31] = m2;
    K[32] = m3;
    K[33] = m4;
    K[34] = m4;
    K[35] = m5;
    K[36] = m5;
    K[37] = m6;
    K[38] = m5;
    K[39] = m0;
    K[40] = m1;
    K[41] = m4;
    K[42] = m4;
    K[43] = m3;
    K[44] = m2;
    K[45] = m4;
    K[46] = m4;
    K[47] = m3;
    K[48] = m2;
    K[49] = m4;
    K[50] = m4;
    K[51] = m2;
    K[52] = m3;
    K[53] = m5;
    K[54] = m6;
    K[55] = m5;
    K[56] = m5;
    K[57] = m0;
    K[58] = m4;
    K[59] = m4;
    K[60] = m4;
    K[61] = m4;
    K[62] = m3;
    K[63] = m2;
    K[64] = m4;
    K[65] = m4;
    K[66] = m3;
    K[67] = m2;
    K[68] = m3;
    K[69] = m2;
    K[70] = m6;
    K[71] = m5;
    K[72] = m5;
    K[73] = m5;
    K[74] = m7;
    K[75] = m8;
    K[76] = m9;
    K[77] = m10;
    K[78] = m9;
    K[79] = m10;
    K[80] = m10;
    K[81] = Ops::zero();
    K[82] = m10;
    K[83] = Ops::zero();
    K[84] = Ops::zero();
    K[85] = Ops::zero();
    K[86] = Ops::zero();
    K[87] = Ops::zero();
    K[88] = Ops::zero();
    K[89] = m8;
    K[90] = m7;
    K[91] = m10;
    K[92] = Ops::zero();
    K[93] = m10;
    K[94] = Ops::zero();
    K[95] = m9;
    K[96] = m10;
    K[97] = m9;
    K[98] = m10;
    K[99] = Ops::zero();
    K[100] = Ops::zero();
    K[101] = Ops::zero();
    K[102] = Ops::zero();
    K[103] = m8;
    K[104] = Ops::zero();
    K[105] = m7;
    K[106] = m8;
    K[107] = m9;
    K[108] = m10;
    K[109] = Ops::zero();
    K[110] = m10;
    K[111] = Ops::zero();
    K[112] = Ops::zero();
    K[113] = m10;
    K[114] = Ops::zero();
    K[115] = Ops::zero();
    K[116] = Ops::zero();
    K[117] = Ops::zero();
    K[118] = m8;
    K[119] = m7;
    K[120] = m10;
    K[121] = Ops::zero();
    K[122] = m10;
    K[123] = m9;
    K[124] = Ops::zero();
    K[125] = Ops::zero();
    K[126] = m9;
    K[127] = m10;
    K[128] = Ops::zero();
    K[129] = m8;
    K[130] = Ops::zero();
    K[131] = Ops::zero();
    K[132] = m7;
    K[133] = m8;
    K[134] = Ops::zero();
    K[135] = Ops::zero();
    K[136] = Ops::zero();
    K[137] = m10;
    K[138] = Ops::zero();
    K[139] = m10;
    K[140] = Ops::zero();
    K[141] = Ops::zero();
    K[142] = Ops::zero();
    K[143] = m8;
    K[144] = m7;
    K[145] = Ops::zero();
    K[146] = Ops::zero();
    K[147] = m10;
    K[148] = m9;
    K[149] = m10;
    K[150] = m9;
    K[151] = m8;
    K[152] = Ops::zero();
    K[153] = Ops::zero();
    K[154] = Ops::zero();
    K[155] = m7;
    K[156] = m8;
    K[157] = m9;
    K[158] = m10;
    K[159] = m10;
    K[160] = Ops::zero();
    K[161] = Ops::zero();
    K[162] = Ops::zero();
    K[163] = m8;
    K[164] = Ops::zero();
    K[165] = m7;
    K[166] = m10;
    K[167] = Ops::zero();
    K[168] = m9;
    K[169] = m10;
    K[170] = Ops::zero();
    K[171] = m8;
    K[172] = Ops::zero();
    K[173] = Ops::zero();
    K[174] = m7;
    K[175] = m8;
    K[176] = Ops::zero();
    K[177] = m10;
    K[178] = Ops::zero();
    K[179] = Ops::zero();
    K[180] = m8;
    K[181] = Ops::zero();
    K[182] = m7;
    K[183] = m10;
    K[184] = m9;
    K[185] = m8;
    K[186] = Ops::zero();
    K[187] = Ops::zero();
    K[188] = Ops::zero();
    K[189] = m7;
    K[190] = m8;
    K[191] = Ops::zero();
    K[192] = m8;
    K[193] = Ops::zero();
    K[194] = Ops::zero();
    K[195] = m7;
    K[196] = m8;
    K[197] = Ops::zero();
    K[198] = Ops::zero();
    K[199] = Ops::zero();
    K[200] = m11;
    K[201] = m12;
    K[202] = m12;
    K[203] = m12;
    K[204] = m11;
    K[205] = m12;
    K[206] = m12;
    K[207] = m11;
    K[208] = m12;
    K[209] = m11;
  }
  template <class Ops, bool STIFF, bool MASS> __device__ __forceinline__ static void action_upper(const typename Ops::T* Lam, const typename Ops::T& vol, const typename Ops::T* x, typename Ops::T* y) {
    typename Ops::T k;
    if constexpr (STIFF && MASS) {
      const typename Ops::T w0 = Ops::add(Lam[1], Lam[2]);
      const typename Ops::T w1 = Ops::add(Lam[3], Lam[6]);
      const typename Ops::T w2 = Ops::add(Lam[5], Lam[8]);
      const typename Ops::T w3 = Ops::add(Lam[0], Lam[3]);
      const typename Ops::T w4 = Ops::add(Lam[1], Lam[4]);
      const typename Ops::T w5 = Ops::add(Lam[2], Lam[7]);
      const typename Ops::T w6 = Ops::add(Lam[8], Lam[9]);
      const typename Ops::T w7 = Ops::add(Lam[5], Lam[6]);
      const typename Ops::T w8 = Ops::add(Lam[1], Lam[3]);
      const typename Ops::T w9 = Ops::add(Lam[2], Lam[5]);
      const typename Ops::T w10 = Ops::add(Lam[6], Lam[8]);
      const typename Ops::T w11 = Ops::add(Lam[1], Lam[5]);
      const typename Ops::T w12 = Ops::add(Lam[1], Lam[6]);
      const typename Ops::T w13 = Ops::add(Lam[2], Lam[3]);
      const typename Ops::T w14 = Ops::add(Lam[2], Lam[8]);
      const typename Ops::T w15 = Ops::add(Lam[3], Lam[8]);
      const typename Ops::T w16 = Ops::add(Lam[0], w0);
      const typename Ops::T w17 = Ops::add(Lam[4], Lam[5]);
      const typename Ops::T w18 = Ops::add(Lam[4], Lam[6]);
      const typename Ops::T w19 = Ops::add(Lam[7], w2);
      const typename Ops::T w20 = Ops::add(Lam[9], w1);
      const typename Ops::T w21 = Ops::add(Lam[0], Lam[1]);
      const typename Ops::T w22 = Ops::add(Lam[0], Lam[2]);
      const typename Ops::T w23 = Ops::add(Lam[3], Lam[9]);
      const typename Ops::T w24 = Ops::add(Lam[5], Lam[7]);
      const typename Ops::T w25 = Ops::add(Lam[6], Lam[9]);
      const typename Ops::T w26 = Ops::add(Lam[7], Lam[8]);
      const typename Ops::T w27 = Ops::add(w0, w3);
      const typename Ops::T w28 = Ops::add(w0, w10);
      const typename Ops::T w29 = Ops::add(w1, w6);
      const typename Ops::T w30 = Ops::add(w1, w9);
      const typename Ops::T w31 = Ops::add(w2, w5);
      const typename Ops::T w32 = Ops::add(w2, w8);
      const typename Ops::T w33 = Ops::add(Lam[1], w3);
      const typename Ops::T w34 = Ops::add(Lam[2], w3);
      const typename Ops::T w35 = Ops::add(Lam[3], w6);
      const typename Ops::T w36 = Ops::add(Lam[4], w7);
      const typename Ops::T w37 = Ops::add(Lam[5], w4);
      const typename Ops::T w38 = Ops::add(Lam[5], w5);
      const typename Ops::T w39 = Ops::add(Lam[6], w4);
      const typename Ops::T w40 = Ops::add(Lam[6], w6);
      const typename Ops::T w41 = Ops::add(Lam[8], w5);
      const typename Ops::T w42 = Ops::add(w4, w7);
      const typename Ops::T w43 = Ops::fmac(Lam[1], -5.0, Lam[0]);
      const typename Ops::T w44 = Ops::fmac(Lam[2], -5.0, Lam[0]);
      const typename Ops::T w45 = Ops::fmac(Lam[3], -5.0, Lam[0]);
      const typename Ops::T w46 = Ops::fmac(Lam[4], -0.2, Lam[1]);
      const typename Ops::T w47 = Ops::fmac(w20, 0.5, Lam[1]);
      const typename Ops::T w48 = Ops::fmac(Lam[7], -0.2, Lam[2]);
      const typename Ops::T w49 = Ops::fmac(Lam[9], -0.2, Lam[3]);
      const typename Ops::T w50 = Ops::fmac(Lam[5], -5.0, Lam[4]);
      const typename Ops::T w51 = Ops::fmac(Lam[6], -5.0, Lam[4]);
      const typename Ops::T w52 = Ops::fmac(Lam[7], -0.2, Lam[5]);
      const typename Ops::T w53 = Ops::fmac(w16, 0.5, Lam[5]);
      const typename Ops::T w54 = Ops::fmac(Lam[9], -0.2, Lam[6]);
      const typename Ops::T w55 = Ops::fmac(w19, 0.5, Lam[6]);
      const typename Ops::T w56 = Ops::fmac(Lam[8], -5.0, Lam[7]);
      const typename Ops::T w57 = Ops::fmac(Lam[9], -0.2, Lam[8]);
      const typename Ops::T w58 = Ops::add(w4, w20);
      const typename Ops::T w59 = Ops::add(w16, w17);
      const typename Ops::T w60 = Ops::add(w18, w19);
      const typename Ops::T m0 = Ops::mulc(vol, 0.0035714285714285713);
      const typename Ops::T m1 = Ops::mulc(vol, 0.0004464285714285714);
      const typename Ops::T m2 = Ops::mulc(vol, -0.0026785714285714286);
      const typename Ops::T m3 = Ops::mulc(vol, 0.0013392857142857143);
      const typename Ops::T m4 = Ops::mulc(vol, 0.0006696428571428571);
      const typename Ops::T m5 = Ops::mulc(vol, 0.0040178571428571425);
      const typename Ops::T m6 = Ops::mulc(vol, 0.008035714285714285);
      const typename Ops::T m7 = Ops::mulc(vol, 0.024107142857142858);
      const typename Ops::T m8 = Ops::mulc(vol, -0.012053571428571429);
      const typename Ops::T m9 = Ops::mulc(vol, 0.012053571428571429);
      const typename Ops::T m10 = Ops::mulc(vol, -0.0060267857142857146);
      const typename Ops::T m11 = Ops::mulc(vol, 0.09642857142857143);
      const typename Ops::T m12 = Ops::mulc(vol, 0.048214285714285716);
      { k = Ops::fmac(Lam[0], 0.35714285714285715, m0); y[0] = Ops::mul(k, x[0]); }
      { k = Ops::fmac(Lam[1], 0.06785714285714285, m1); y[0] = Ops::fma3(k, x[1], y[0]); y[1] = Ops::mul(k, x[0]); }
      { k = Ops::fmac(Lam[2], 0.06785714285714285, m1); y[0] = Ops::fma3(k, x[2], y[0]); y[2] = Ops::mul(k, x[0]); }
      { k = Ops::fmac(Lam[3], 0.06785714285714285, m1); y[0] = Ops::fma3(k, x[3], y[0]); y[3] = Ops::mul(k, x[0]); }
      { k = Ops::fmac(Lam[1], 0.36964285714285716, Ops::fmac(Lam[0], -0.20892857142857144, m2)); y[0] = Ops::fma3(k, x[4], y[0]); y[4] = Ops::mul(k, x[0]); }
      { k = Ops::fmac(Lam[1], -0.20892857142857144, Ops::fmac(Lam[0], 0.08035714285714286, m3)); y[0] = Ops::fma3(k, x[5], y[0]); y[5] = Ops::mul(k, x[0]); }
      { k = Ops::fmac(Lam[2], 0.36964285714285716, Ops::fmac(Lam[0], -0.20892857142857144, m2)); y[0] = Ops::fma3(k, x[6], y[0]); y[6] = Ops::mul(k, x[0]); }
      { k = Ops::fmac(Lam[2], -0.20892857142857144, Ops::fmac(Lam[0], 0.08035714285714286, m3)); y[0] = Ops::fma3(k, x[7], y[0]); y[7] = Ops::mul(k, x[0]); }
      { k = Ops::fmac(Lam[3], 0.36964285714285716, Ops::fmac(Lam[0], -0.20892857142857144, m2)); y[0] = Ops::fma3(k, x[8], y[0]); y[8] = Ops::mul(k, x[0]); }
      { k = Ops::fmac(Lam[3], -0.20892857142857144, Ops::fmac(Lam[0], 0.08035714285714286, m3)); y[0] = Ops::fma3(k, x[9], y[0]); y[9] = Ops::mul(k, x[0]); }
      { k = Ops::fmac(w0, 0.08035714285714286, m4); y[0] = Ops::fma3(k, x[10], y[0]); y[10] = Ops::mul(k, x[0]); }
      { k = Ops::fmac(w0, 0.08035714285714286, m4); y[0] = Ops::fma3(k, x[11], y[0]); y[11] = Ops::mul(k, x[0]); }
      { k = Ops::fmac(w8, 0.08035714285714286, m4); y[0] = Ops::fma3(k, x[12], y[0]); y[12] = Ops::mul(k, x[0]); }
      { k = Ops::fmac(w8, 0.08035714285714286, m4); y[0] = Ops::fma3(k, x[13], y[0]); y[13] = Ops::mul(k, x[0]); }
      { k = Ops::fmac(w13, 0.08035714285714286, m4); y[0] = Ops::fma3(k, x[14], y[0]); y[14] = Ops::mul(k, x[0]); }
      { k = Ops::fmac(w13, 0.08035714285714286, m4); y[0] = Ops::fma3(k, x[15], y[0]); y[15] = Ops::mul(k, x[0]); }
      { k = Ops::fmac(w0, -0.09642857142857143, Ops::fmac(Lam[0], 0.19285714285714287, m5)); y[0] = Ops::fma3(k, x[16], y[0]); y[16] = Ops::mul(k, x[0]); }
      { k = Ops::fmac(w8, -0.09642857142857143, Ops::fmac(Lam[0], 0.19285714285714287, m5)); y[0] = Ops::fma3(k, x[17], y[0]); y[17] = Ops::mul(k, x[0]); }
      { k = Ops::fmac(w13, -0.09642857142857143, Ops::fmac(Lam[0], 0.19285714285714287, m5)); y[0] = Ops::fma3(k, x[18], y[0]); y[18] = Ops::mul(k, x[0]); }
      { k = Ops::fmac(w0, 0.19285714285714287, Ops::fmac(Lam[3], 0.19285714285714287, m6)); y[0] = Ops::fma3(k, x[19], y[0]); y[19] = Ops::mul(k, x[0]); }
      { k = Ops::fmac(Lam[4], 0.35714285714285715, m0); y[1] = Ops::fma3(k, x[1], y[1]); }
      { k = Ops::fmac(Lam[5], 0.06785714285714285, m1); y[1] = Ops::fma3(k, x[2], y[1]); y[2] = Ops::fma3(k, x[1], y[2]); }
      { k = Ops::fmac(Lam[6], 0.06785714285714285, m1); y[1] = Ops::fma3(k, x[3], y[1]); y[3] = Ops::fma3(k, x[1], y[3]); }
      { k = Ops::fmac(Lam[4], 0.08035714285714286, Ops::fmac(Lam[1], -0.20892857142857144, m3)); y[1] = Ops::fma3(k, x[4], y[1]); y[4] = Ops::fma3(k, x[1], y[4]); }
      { k = Ops::fmac(Lam[4], -0.20892857142857144, Ops::fmac(Lam[1], 0.36964285714285716, m2)); y[1] = Ops::fma3(k, x[5], y[1]); y[5] = Ops::fma3(k, x[1], y[5]); }
      { k = Ops::fmac(w11, 0.08035714285714286, m4); y[1] = Ops::fma3(k, x[6], y[1]); y[6] = Ops::fma3(k, x[1], y[6]); }
      { k = Ops::fmac(w11, 0.08035714285714286, m4); y[1] = Ops::fma3(k, x[7], y[1]); y[7] = Ops::fma3(k, x[1], y[7]); }
      { k = Ops::fmac(w12, 0.08035714285714286, m4); y[1] = Ops::fma3(k, x[8], y[1]); y[8] = Ops::fma3(k, x[1], y[8]); }
      { k = Ops::fmac(w12, 0.08035714285714286, m4); y[1] = Ops::fma3(k, x[9], y[1]); y[9] = Ops::fma3(k, x[1], y[9]); }
      { k = Ops::fmac(Lam[5], 0.36964285714285716, Ops::fmac(Lam[4], -0.20892857142857144, m2)); y[1] = Ops::fma3(k, x[10], y[1]); y[10] = Ops::fma3(k, x[1], y[10]); }
      { k = Ops::fmac(Lam[5], -0.20892857142857144, Ops::fmac(Lam[4], 0.08035714285714286, m3)); y[1] = Ops::fma3(k, x[11], y[1]); y[11] = Ops::fma3(k, x[1], y[11]); }
      { k = Ops::fmac(Lam[6], 0.36964285714285716, Ops::fmac(Lam[4], -0.20892857142857144, m2)); y[1] = Ops::fma3(k, x[12], y[1]); y[12] = Ops::fma3(k, x[1], y[12]); }
      { k = Ops::fmac(Lam[6], -0.20892857142857144, Ops::fmac(Lam[4], 0.08035714285714286, m3)); y[1] = Ops::fma3(k, x[13], y[1]); y[13] = Ops::fma3(k, x[1], y[13]); }
      { k = Ops::fmac(w7, 0.08035714285714286, m4); y[1] = Ops::fma3(k, x[14], y[1]); y[14] = Ops::fma3(k, x[1], y[14]); }
      { k = Ops::fmac(w7, 0.08035714285714286, m4); y[1] = Ops::fma3(k, x[15], y[1]); y[15] = Ops::fma3(k, x[1], y[15]); }
      { k = Ops::fmac(w11, -0.09642857142857143, Ops::fmac(Lam[4], 0.19285714285714287, m5)); y[1] = Ops::fma3(k, x[16], y[1]); y[16] = Ops::fma3(k, x[1], y[16]); }
      { k = Ops::fmac(w12, -0.09642857142857143, Ops::fmac(Lam[4], 0.19285714285714287, m5)); y[1] = Ops::fma3(k, x[17], y[1]); y[17] = Ops::fma3(k, x[1], y[17]); }
      { k = Ops::fmac(w7, 0.19285714285714287, Ops::fmac(Lam[1], 0.19285714285714287, m6)); y[1] = Ops::fma3(k, x[18], y[1]); y[18] = Ops::fma3(k, x[1], y[18]); }
      { k = Ops::fmac(w7, -0.09642857142857143, Ops::fmac(Lam[4], 0.19285714285714287, m5)); y[1] = Ops::fma3(k, x[19], y[1]); y[19] = Ops::fma3(k, x[1], y[19]); }
      { k = Ops::fmac(Lam[7], 0.35714285714285715, m0); y[2] = Ops::fma3(k, x[2], y[2]); }
      { k = Ops::fmac(Lam[8], 0.06785714285714285, m1); y[2] = Ops::fma3(k, x[3], y[2]); y[3] = Ops::fma3(k, x[2], y[3]); }
      { k = Ops::fmac(w9, 0.08035714285714286, m4); y[2] = Ops::fma3(k, x[4], y[2]); y[4] = Ops::fma3(k, x[2], y[4]); }
      { k = Ops::fmac(w9, 0.08035714285714286, m4); y[2] = Ops::fma3(k, x[5], y[2]); y[5] = Ops::fma3(k, x[2], y[5]); }
      { k = Ops::fmac(Lam[7], 0.08035714285714286, Ops::fmac(Lam[2], -0.20892857142857144, m3)); y[2] = Ops::fma3(k, x[6], y[2]); y[6] = Ops::fma3(k, x[2], y[6]); }
      { k = Ops::fmac(Lam[7], -0.20892857142857144, Ops::fmac(Lam[2], 0.36964285714285716, m2)); y[2] = Ops::fma3(k, x[7], y[2]); y[7] = Ops::fma3(k, x[2], y[7]); }
      { k = Ops::fmac(w14, 0.08035714285714286, m4); y[2] = Ops::fma3(k, x[8], y[2]); y[8] = Ops::fma3(k, x[2], y[8]); }
      { k = Ops::fmac(w14, 0.08035714285714286, m4); y[2] = Ops::fma3(k, x[9], y[2]); y[9] = Ops::fma3(k, x[2], y[9]); }
      { k = Ops::fmac(Lam[7], 0.08035714285714286, Ops::fmac(Lam[5], -0.20892857142857144, m3)); y[2] = Ops::fma3(k, x[10], y[2]); y[10] = Ops::fma3(k, x[2], y[10]); }
      { k = Ops::fmac(Lam[7], -0.20892857142857144, Ops::fmac(Lam[5], 0.36964285714285716, m2)); y[2] = Ops::fma3(k, x[11], y[2]); y[11] = Ops::fma3(k, x[2], y[11]); }
      { k = Ops::fmac(w2, 0.08035714285714286, m4); y[2] = Ops::fma3(k, x[12], y[2]); y[12] = Ops::fma3(k, x[2], y[12]); }
      { k = Ops::fmac(w2, 0.08035714285714286, m4); y[2] = Ops::fma3(k, x[13], y[2]); y[13] = Ops::fma3(k, x[2], y[13]); }
      { k = Ops::fmac(Lam[8], 0.36964285714285716, Ops::fmac(Lam[7], -0.20892857142857144, m2)); y[2] = Ops::fma3(k, x[14], y[2]); y[14] = Ops::fma3(k, x[2], y[14]); }
      { k = Ops::fmac(Lam[8], -0.20892857142857144, Ops::fmac(Lam[7], 0.08035714285714286, m3)); y[2] = Ops::fma3(k, x[15], y[2]); y[15] = Ops::fma3(k, x[2], y[15]); }
      { k = Ops::fmac(w9, -0.09642857142857143, Ops::fmac(Lam[7], 0.19285714285714287, m5)); y[2] = Ops::fma3(k, x[16], y[2]); y[16] = Ops::fma3(k, x[2], y[16]); }
      { k = Ops::fmac(w2, 0.19285714285714287, Ops::fmac(Lam[2], 0.19285714285714287, m6)); y[2] = Ops::fma3(k, x[17], y[2]); y[17] = Ops::fma3(k, x[2], y[17]); }
      { k = Ops::fmac(w14, -0.09642857142857143, Ops::fmac(Lam[7], 0.19285714285714287, m5)); y[2] = Ops::fma3(k, x[18], y[2]); y[18] = Ops::fma3(k, x[2], y[18]); }
      { k = Ops::fmac(w2, -0.09642857142857143, Ops::fmac(Lam[7], 0.19285714285714287, m5)); y[2] = Ops::fma3(k, x[19], y[2]); y[19] = Ops::fma3(k, x[2], y[19]); }
      { k = Ops::fmac(Lam[9], 0.35714285714285715, m0); y[3] = Ops::fma3(k, x[3], y[3]); }
      { k = Ops::fmac(w1, 0.08035714285714286, m4); y[3] = Ops::fma3(k, x[4], y[3]); y[4] = Ops::fma3(k, x[3], y[4]); }
      { k = Ops::fmac(w1, 0.08035714285714286, m4); y[3] = Ops::fma3(k, x[5], y[3]); y[5] = Ops::fma3(k, x[3], y[5]); }
      { k = Ops::fmac(w15, 0.08035714285714286, m4); y[3] = Ops::fma3(k, x[6], y[3]); y[6] = Ops::fma3(k, x[3], y[6]); }
      { k = Ops::fmac(w15, 0.08035714285714286, m4); y[3] = Ops::fma3(k, x[7], y[3]); y[7] = Ops::fma3(k, x[3], y[7]); }
      { k = Ops::fmac(Lam[9], 0.08035714285714286, Ops::fmac(Lam[3], -0.20892857142857144, m3)); y[3] = Ops::fma3(k, x[8], y[3]); y[8] = Ops::fma3(k, x[3], y[8]); }
      { k = Ops::fmac(Lam[9], -0.20892857142857144, Ops::fmac(Lam[3], 0.36964285714285716, m2)); y[3] = Ops::fma3(k, x[9], y[3]); y[9] = Ops::fma3(k, x[3], y[9]); }
      { k = Ops::fmac(w10, 0.08035714285714286, m4); y[3] = Ops::fma3(k, x[10], y[3]); y[10] = Ops::fma3(k, x[3], y[10]); }
      { k = Ops::fmac(w10, 0.08035714285714286, m4); y[3] = Ops::fma3(k, x[11], y[3]); y[11] = Ops::fma3(k, x[3], y[11]); }
      { k = Ops::fmac(Lam[9], 0.08035714285714286, Ops::fmac(Lam[6], -0.20892857142857144, m3)); y[3] = Ops::fma3(k, x[12], y[3]); y[12] = Ops::fma3(k, x[3], y[12]); }
      { k = Ops::fmac(Lam[9], -0.20892857142857144, Ops::fmac(Lam[6], 0.36964285714285716, m2)); y[3] = Ops::fma3(k, x[13], y[3]); y[13] = Ops::fma3(k, x[3], y[13]); }
      { k = Ops::fmac(Lam[9], 0.08035714285714286, Ops::fmac(Lam[8], -0.20892857142857144, m3)); y[3] = Ops::fma3(k, x[14], y[3]); y[14] = Ops::fma3(k, x[3], y[14]); }
      { k = Ops::fmac(Lam[9], -0.20892857142857144, Ops::fmac(Lam[8], 0.36964285714285716, m2)); y[3] = Ops::fma3(k, x[15], y[3]); y[15] = Ops::fma3(k, x[3], y[15]); }
      { k = Ops::fmac(w1, 0.19285714285714287, Ops::fmac(Lam[8], 0.19285714285714287, m6)); y[3] = Ops::fma3(k, x[16], y[3]); y[16] = Ops::fma3(k, x[3], y[16]); }
      { k = Ops::fmac(w1, -0.09642857142857143, Ops::fmac(Lam[9], 0.19285714285714287, m5)); y[3] = Ops::fma3(k, x[17], y[3]); y[17] = Ops::fma3(k, x[3], y[17]); }
      { k = Ops::fmac(w15, -0.09642857142857143, Ops::fmac(Lam[9], 0.19285714285714287, m5)); y[3] = Ops::fma3(k, x[18], y[3]); y[18] = Ops::fma3(k, x[3], y[18]); }
      { k = Ops::fmac(w10, -0.09642857142857143, Ops::fmac(Lam[9], 0.19285714285714287, m5)); y[3] = Ops::fma3(k, x[19], y[3]); y[19] = Ops::fma3(k, x[3], y[19]); }
      { k = Ops::fmac(w4, 1.1571428571428573, Ops::fmac(Lam[0], 1.4464285714285714, m7)); y[4] = Ops::fma3(k, x[4], y[4]); }
      { k = Ops::fmac(Lam[4], -0.43392857142857144, Ops::fmac(Lam[1], 0.2892857142857143, Ops::fmac(Lam[0], -0.43392857142857144, m8))); y[4] = Ops::fma3(k, x[5], y[4]); y[5] = Ops::fma3(k, x[4], y[5]); }
      { k = Ops::fmac(w0, 0.5785714285714286, Ops::fmac(Lam[5], 1.1571428571428573, Ops::fmac(Lam[0], 0.7232142857142857, m9))); y[4] = Ops::fma3(k, x[6], y[4]); y[6] = Ops::fma3(k, x[4], y[6]); }
      { k = Ops::fmac(w21, -0.14464285714285716, Ops::fmac(Lam[5], -0.43392857142857144, Ops::fmac(Lam[2], -0.2892857142857143, m10))); y[4] = Ops::fma3(k, x[7], y[4]); y[7] = Ops::fma3(k, x[4], y[7]); }
      { k = Ops::fmac(w8, 0.5785714285714286, Ops::fmac(Lam[6], 1.1571428571428573, Ops::fmac(Lam[0], 0.7232142857142857, m9))); y[4] = Ops::fma3(k, x[8], y[4]); y[8] = Ops::fma3(k, x[4], y[8]); }
      { k = Ops::fmac(w21, -0.14464285714285716, Ops::fmac(Lam[6], -0.43392857142857144, Ops::fmac(Lam[3], -0.2892857142857143, m10))); y[4] = Ops::fma3(k, x[9], y[4]); y[9] = Ops::fma3(k, x[4], y[9]); }
      { k = Ops::fmac(w17, -0.14464285714285716, Ops::fmac(Lam[2], -0.43392857142857144, Ops::fmac(Lam[1], -0.2892857142857143, m10))); y[4] = Ops::fma3(k, x[10], y[4]); y[10] = Ops::fma3(k, x[4], y[10]); }
      { k = Ops::fmac(w37, -0.14464285714285716, Ops::mulc(Lam[2], -0.2892857142857143)); y[4] = Ops::fma3(k, x[11], y[4]); y[11] = Ops::fma3(k, x[4], y[11]); }
      { k = Ops::fmac(w18, -0.14464285714285716, Ops::fmac(Lam[3], -0.43392857142857144, Ops::fmac(Lam[1], -0.2892857142857143, m10))); y[4] = Ops::fma3(k, x[12], y[4]); y[12] = Ops::fma3(k, x[4], y[12]); }
      { k = Ops::fmac(w39, -0.14464285714285716, Ops::mulc(Lam[3], -0.2892857142857143)); y[4] = Ops::fma3(k, x[13], y[4]); y[13] = Ops::fma3(k, x[4], y[13]); }
      { k = Ops::mulc(w30, -0.14464285714285716); y[4] = Ops::fma3(k, x[14], y[4]); y[14] = Ops::fma3(k, x[4], y[14]); }
      { k = Ops::mulc(w30, -0.14464285714285716); y[4] = Ops::fma3(k, x[15], y[4]); y[15] = Ops::fma3(k, x[4], y[15]); }
      { k = Ops::fmac(w44, -0.2892857142857143, Ops::mulc(w37, 0.5785714285714286)); y[4] = Ops::fma3(k, x[16], y[4]); y[16] = Ops::fma3(k, x[4], y[16]); }
      { k = Ops::fmac(w45, -0.2892857142857143, Ops::mulc(w39, 0.5785714285714286)); y[4] = Ops::fma3(k, x[17], y[4]); y[17] = Ops::fma3(k, x[4], y[17]); }
      { k = Ops::fmac(w21, -0.14464285714285716, Ops::fmac(w13, 0.7232142857142857, Ops::mulc(w7, 0.5785714285714286))); y[4] = Ops::fma3(k, x[18], y[4]); y[18] = Ops::fma3(k, x[4], y[18]); }
      { k = Ops::fmac(w42, -0.14464285714285716, Ops::fmac(w13, -0.2892857142857143, m8)); y[4] = Ops::fma3(k, x[19], y[4]); y[19] = Ops::fma3(k, x[4], y[19]); }
      { k = Ops::fmac(w21, 1.1571428571428573, Ops::fmac(Lam[4], 1.4464285714285714, m7)); y[5] = Ops::fma3(k, x[5], y[5]); }
      { k = Ops::fmac(w22, -0.14464285714285716, Ops::fmac(Lam[5], -0.43392857142857144, Ops::fmac(Lam[1], -0.2892857142857143, m10))); y[5] = Ops::fma3(k, x[6], y[5]); y[6] = Ops::fma3(k, x[5], y[6]); }
      { k = Ops::mulc(w53, -0.2892857142857143); y[5] = Ops::fma3(k, x[7], y[5]); y[7] = Ops::fma3(k, x[5], y[7]); }
      { k = Ops::fmac(w3, -0.14464285714285716, Ops::fmac(Lam[6], -0.43392857142857144, Ops::fmac(Lam[1], -0.2892857142857143, m10))); y[5] = Ops::fma3(k, x[8], y[5]); y[8] = Ops::fma3(k, x[5], y[8]); }
      { k = Ops::fmac(w33, -0.14464285714285716, Ops::mulc(Lam[6], -0.2892857142857143)); y[5] = Ops::fma3(k, x[9], y[5]); y[9] = Ops::fma3(k, x[5], y[9]); }
      { k = Ops::fmac(w11, 0.5785714285714286, Ops::fmac(Lam[4], 0.7232142857142857, Ops::fmac(Lam[2], 1.1571428571428573, m9))); y[5] = Ops::fma3(k, x[10], y[5]); y[10] = Ops::fma3(k, x[5], y[10]); }
      { k = Ops::fmac(w4, -0.14464285714285716, Ops::fmac(Lam[5], -0.2892857142857143, Ops::fmac(Lam[2], -0.43392857142857144, m10))); y[5] = Ops::fma3(k, x[11], y[5]); y[11] = Ops::fma3(k, x[5], y[11]); }
      { k = Ops::fmac(w12, 0.5785714285714286, Ops::fmac(Lam[4], 0.7232142857142857, Ops::fmac(Lam[3], 1.1571428571428573, m9))); y[5] = Ops::fma3(k, x[12], y[5]); y[12] = Ops::fma3(k, x[5], y[12]); }
      { k = Ops::fmac(w4, -0.14464285714285716, Ops::fmac(Lam[6], -0.2892857142857143, Ops::fmac(Lam[3], -0.43392857142857144, m10))); y[5] = Ops::fma3(k, x[13], y[5]); y[13] = Ops::fma3(k, x[5], y[13]); }
      { k = Ops::mulc(w30, -0.14464285714285716); y[5] = Ops::fma3(k, x[14], y[5]); y[14] = Ops::fma3(k, x[5], y[14]); }
      { k = Ops::mulc(w30, -0.14464285714285716); y[5] = Ops::fma3(k, x[15], y[5]); y[15] = Ops::fma3(k, x[5], y[15]); }
      { k = Ops::fmac(w50, -0.2892857142857143, Ops::mulc(w16, 0.5785714285714286)); y[5] = Ops::fma3(k, x[16], y[5]); y[16] = Ops::fma3(k, x[5], y[16]); }
      { k = Ops::fmac(w51, -0.2892857142857143, Ops::mulc(w33, 0.5785714285714286)); y[5] = Ops::fma3(k, x[17], y[5]); y[17] = Ops::fma3(k, x[5], y[17]); }
      { k = Ops::fmac(w27, -0.14464285714285716, Ops::fmac(w7, -0.2892857142857143, m8)); y[5] = Ops::fma3(k, x[18], y[5]); y[18] = Ops::fma3(k, x[5], y[18]); }
      { k = Ops::fmac(w13, 0.5785714285714286, Ops::fmac(w7, 0.7232142857142857, Ops::mulc(w4, -0.14464285714285716))); y[5] = Ops::fma3(k, x[19], y[5]); y[19] = Ops::fma3(k, x[5], y[19]); }
      { k = Ops::fmac(w5, 1.1571428571428573, Ops::fmac(Lam[0], 1.4464285714285714, m7)); y[6] = Ops::fma3(k, x[6], y[6]); }
      { k = Ops::fmac(Lam[7], -0.43392857142857144, Ops::fmac(Lam[2], 0.2892857142857143, Ops::fmac(Lam[0], -0.43392857142857144, m8))); y[6] = Ops::fma3(k, x[7], y[6]); y[7] = Ops::fma3(k, x[6], y[7]); }
      { k = Ops::fmac(w13, 0.5785714285714286, Ops::fmac(Lam[8], 1.1571428571428573, Ops::fmac(Lam[0], 0.7232142857142857, m9))); y[6] = Ops::fma3(k, x[8], y[6]); y[8] = Ops::fma3(k, x[6], y[8]); }
      { k = Ops::fmac(w22, -0.14464285714285716, Ops::fmac(Lam[8], -0.43392857142857144, Ops::fmac(Lam[3], -0.2892857142857143, m10))); y[6] = Ops::fma3(k, x[9], y[6]); y[9] = Ops::fma3(k, x[6], y[9]); }
      { k = Ops::fmac(w38, -0.14464285714285716, Ops::mulc(Lam[1], -0.2892857142857143)); y[6] = Ops::fma3(k, x[10], y[6]); y[10] = Ops::fma3(k, x[6], y[10]); }
      { k = Ops::fmac(w24, -0.14464285714285716, Ops::fmac(Lam[2], -0.2892857142857143, Ops::fmac(Lam[1], -0.43392857142857144, m10))); y[6] = Ops::fma3(k, x[11], y[6]); y[11] = Ops::fma3(k, x[6], y[11]); }
      { k = Ops::mulc(w32, -0.14464285714285716); y[6] = Ops::fma3(k, x[12], y[6]); y[12] = Ops::fma3(k, x[6], y[12]); }
      { k = Ops::mulc(w32, -0.14464285714285716); y[6] = Ops::fma3(k, x[13], y[6]); y[13] = Ops::fma3(k, x[6], y[13]); }
      { k = Ops::fmac(w26, -0.14464285714285716, Ops::fmac(Lam[3], -0.43392857142857144, Ops::fmac(Lam[2], -0.2892857142857143, m10))); y[6] = Ops::fma3(k, x[14], y[6]); y[14] = Ops::fma3(k, x[6], y[14]); }
      { k = Ops::fmac(w41, -0.14464285714285716, Ops::mulc(Lam[3], -0.2892857142857143)); y[6] = Ops::fma3(k, x[15], y[6]); y[15] = Ops::fma3(k, x[6], y[15]); }
      { k = Ops::fmac(w43, -0.2892857142857143, Ops::mulc(w38, 0.5785714285714286)); y[6] = Ops::fma3(k, x[16], y[6]); y[16] = Ops::fma3(k, x[6], y[16]); }
      { k = Ops::fmac(w22, -0.14464285714285716, Ops::fmac(w8, 0.7232142857142857, Ops::mulc(w2, 0.5785714285714286))); y[6] = Ops::fma3(k, x[17], y[6]); y[17] = Ops::fma3(k, x[6], y[17]); }
      { k = Ops::fmac(w45, -0.2892857142857143, Ops::mulc(w41, 0.5785714285714286)); y[6] = Ops::fma3(k, x[18], y[6]); y[18] = Ops::fma3(k, x[6], y[18]); }
      { k = Ops::fmac(w31, -0.14464285714285716, Ops::fmac(w8, -0.2892857142857143, m8)); y[6] = Ops::fma3(k, x[19], y[6]); y[19] = Ops::fma3(k, x[6], y[19]); }
      { k = Ops::fmac(w22, 1.1571428571428573, Ops::fmac(Lam[7], 1.4464285714285714, m7)); y[7] = Ops::fma3(k, x[7], y[7]); }
      { k = Ops::fmac(w3, -0.14464285714285716, Ops::fmac(Lam[8], -0.43392857142857144, Ops::fmac(Lam[2], -0.2892857142857143, m10))); y[7] = Ops::fma3(k, x[8], y[7]); y[8] = Ops::fma3(k, x[7], y[8]); }
      { k = Ops::fmac(w34, -0.14464285714285716, Ops::mulc(Lam[8], -0.2892857142857143)); y[7] = Ops::fma3(k, x[9], y[7]); y[9] = Ops::fma3(k, x[7], y[9]); }
      { k = Ops::fmac(w5, -0.14464285714285716, Ops::fmac(Lam[5], -0.2892857142857143, Ops::fmac(Lam[1], -0.43392857142857144, m10))); y[7] = Ops::fma3(k, x[10], y[7]); y[10] = Ops::fma3(k, x[7], y[10]); }
      { k = Ops::fmac(w9, 0.5785714285714286, Ops::fmac(Lam[7], 0.7232142857142857, Ops::fmac(Lam[1], 1.1571428571428573, m9))); y[7] = Ops::fma3(k, x[11], y[7]); y[11] = Ops::fma3(k, x[7], y[11]); }
      { k = Ops::mulc(w32, -0.14464285714285716); y[7] = Ops::fma3(k, x[12], y[7]); y[12] = Ops::fma3(k, x[7], y[12]); }
      { k = Ops::mulc(w32, -0.14464285714285716); y[7] = Ops::fma3(k, x[13], y[7]); y[13] = Ops::fma3(k, x[7], y[13]); }
      { k = Ops::fmac(w14, 0.5785714285714286, Ops::fmac(Lam[7], 0.7232142857142857, Ops::fmac(Lam[3], 1.1571428571428573, m9))); y[7] = Ops::fma3(k, x[14], y[7]); y[14] = Ops::fma3(k, x[7], y[14]); }
      { k = Ops::fmac(w5, -0.14464285714285716, Ops::fmac(Lam[8], -0.2892857142857143, Ops::fmac(Lam[3], -0.43392857142857144, m10))); y[7] = Ops::fma3(k, x[15], y[7]); y[15] = Ops::fma3(k, x[7], y[15]); }
      { k = Ops::fmac(w52, 1.4464285714285714, Ops::mulc(w16, 0.5785714285714286)); y[7] = Ops::fma3(k, x[16], y[7]); y[16] = Ops::fma3(k, x[7], y[16]); }
      { k = Ops::fmac(w27, -0.14464285714285716, Ops::fmac(w2, -0.2892857142857143, m8)); y[7] = Ops::fma3(k, x[17], y[7]); y[17] = Ops::fma3(k, x[7], y[17]); }
      { k = Ops::fmac(w56, -0.2892857142857143, Ops::mulc(w34, 0.5785714285714286)); y[7] = Ops::fma3(k, x[18], y[7]); y[18] = Ops::fma3(k, x[7], y[18]); }
      { k = Ops::fmac(w8, 0.5785714285714286, Ops::fmac(w5, -0.14464285714285716, Ops::mulc(w2, 0.7232142857142857))); y[7] = Ops::fma3(k, x[19], y[7]); y[19] = Ops::fma3(k, x[7], y[19]); }
      { k = Ops::fmac(w23, 1.1571428571428573, Ops::fmac(Lam[0], 1.4464285714285714, m7)); y[8] = Ops::fma3(k, x[8], y[8]); }
      { k = Ops::fmac(Lam[9], -0.43392857142857144, Ops::fmac(Lam[3], 0.2892857142857143, Ops::fmac(Lam[0], -0.43392857142857144, m8))); y[8] = Ops::fma3(k, x[9], y[8]); y[9] = Ops::fma3(k, x[8], y[9]); }
      { k = Ops::mulc(w28, -0.14464285714285716); y[8] = Ops::fma3(k, x[10], y[8]); y[10] = Ops::fma3(k, x[8], y[10]); }
      { k = Ops::mulc(w28, -0.14464285714285716); y[8] = Ops::fma3(k, x[11], y[8]); y[11] = Ops::fma3(k, x[8], y[11]); }
      { k = Ops::mulc(w47, -0.2892857142857143); y[8] = Ops::fma3(k, x[12], y[8]); y[12] = Ops::fma3(k, x[8], y[12]); }
      { k = Ops::fmac(w25, -0.14464285714285716, Ops::fmac(Lam[3], -0.2892857142857143, Ops::fmac(Lam[1], -0.43392857142857144, m10))); y[8] = Ops::fma3(k, x[13], y[8]); y[13] = Ops::fma3(k, x[8], y[13]); }
      { k = Ops::fmac(w35, -0.14464285714285716, Ops::mulc(Lam[2], -0.2892857142857143)); y[8] = Ops::fma3(k, x[14], y[8]); y[14] = Ops::fma3(k, x[8], y[14]); }
      { k = Ops::fmac(w6, -0.14464285714285716, Ops::fmac(Lam[3], -0.2892857142857143, Ops::fmac(Lam[2], -0.43392857142857144, m10))); y[8] = Ops::fma3(k, x[15], y[8]); y[15] = Ops::fma3(k, x[8], y[15]); }
      { k = Ops::fmac(w10, 0.5785714285714286, Ops::fmac(w3, -0.14464285714285716, Ops::mulc(w0, 0.7232142857142857))); y[8] = Ops::fma3(k, x[16], y[8]); y[16] = Ops::fma3(k, x[8], y[16]); }
      { k = Ops::fmac(w43, -0.2892857142857143, Ops::mulc(w20, 0.5785714285714286)); y[8] = Ops::fma3(k, x[17], y[8]); y[17] = Ops::fma3(k, x[8], y[17]); }
      { k = Ops::fmac(w44, -0.2892857142857143, Ops::mulc(w35, 0.5785714285714286)); y[8] = Ops::fma3(k, x[18], y[8]); y[18] = Ops::fma3(k, x[8], y[18]); }
      { k = Ops::fmac(w29, -0.14464285714285716, Ops::fmac(w0, -0.2892857142857143, m8)); y[8] = Ops::fma3(k, x[19], y[8]); y[19] = Ops::fma3(k, x[8], y[19]); }
      { k = Ops::fmac(w3, 1.1571428571428573, Ops::fmac(Lam[9], 1.4464285714285714, m7)); y[9] = Ops::fma3(k, x[9], y[9]); }
      { k = Ops::mulc(w28, -0.14464285714285716); y[9] = Ops::fma3(k, x[10], y[9]); y[10] = Ops::fma3(k, x[9], y[10]); }
      { k = Ops::mulc(w28, -0.14464285714285716); y[9] = Ops::fma3(k, x[11], y[9]); y[11] = Ops::fma3(k, x[9], y[11]); }
      { k = Ops::fmac(w23, -0.14464285714285716, Ops::fmac(Lam[6], -0.2892857142857143, Ops::fmac(Lam[1], -0.43392857142857144, m10))); y[9] = Ops::fma3(k, x[12], y[9]); y[12] = Ops::fma3(k, x[9], y[12]); }
      { k = Ops::fmac(w1, 0.5785714285714286, Ops::fmac(Lam[9], 0.7232142857142857, Ops::fmac(Lam[1], 1.1571428571428573, m9))); y[9] = Ops::fma3(k, x[13], y[9]); y[13] = Ops::fma3(k, x[9], y[13]); }
      { k = Ops::fmac(w23, -0.14464285714285716, Ops::fmac(Lam[8], -0.2892857142857143, Ops::fmac(Lam[2], -0.43392857142857144, m10))); y[9] = Ops::fma3(k, x[14], y[9]); y[14] = Ops::fma3(k, x[9], y[14]); }
      { k = Ops::fmac(w15, 0.5785714285714286, Ops::fmac(Lam[9], 0.7232142857142857, Ops::fmac(Lam[2], 1.1571428571428573, m9))); y[9] = Ops::fma3(k, x[15], y[9]); y[15] = Ops::fma3(k, x[9], y[15]); }
      { k = Ops::fmac(w27, -0.14464285714285716, Ops::fmac(w10, -0.2892857142857143, m8)); y[9] = Ops::fma3(k, x[16], y[9]); y[16] = Ops::fma3(k, x[9], y[16]); }
      { k = Ops::fmac(w54, 1.4464285714285714, Ops::mulc(w33, 0.5785714285714286)); y[9] = Ops::fma3(k, x[17], y[9]); y[17] = Ops::fma3(k, x[9], y[17]); }
      { k = Ops::fmac(w57, 1.4464285714285714, Ops::mulc(w34, 0.5785714285714286)); y[9] = Ops::fma3(k, x[18], y[9]); y[18] = Ops::fma3(k, x[9], y[18]); }
      { k = Ops::fmac(w23, -0.14464285714285716, Ops::fmac(w10, 0.7232142857142857, Ops::mulc(w0, 0.5785714285714286))); y[9] = Ops::fma3(k, x[19], y[9]); y[19] = Ops::fma3(k, x[9], y[19]); }
      { k = Ops::fmac(w24, 1.1571428571428573, Ops::fmac(Lam[4], 1.4464285714285714, m7)); y[10] = Ops::fma3(k, x[10], y[10]); }
      { k = Ops::fmac(Lam[7], -0.43392857142857144, Ops::fmac(Lam[5], 0.2892857142857143, Ops::fmac(Lam[4], -0.43392857142857144, m8))); y[10] = Ops::fma3(k, x[11], y[10]); y[11] = Ops::fma3(k, x[10], y[11]); }
      { k = Ops::fmac(w7, 0.5785714285714286, Ops::fmac(Lam[8], 1.1571428571428573, Ops::fmac(Lam[4], 0.7232142857142857, m9))); y[10] = Ops::fma3(k, x[12], y[10]); y[12] = Ops::fma3(k, x[10], y[12]); }
      { k = Ops::fmac(w17, -0.14464285714285716, Ops::fmac(Lam[8], -0.43392857142857144, Ops::fmac(Lam[6], -0.2892857142857143, m10))); y[10] = Ops::fma3(k, x[13], y[10]); y[13] = Ops::fma3(k, x[10], y[13]); }
      { k = Ops::fmac(w26, -0.14464285714285716, Ops::fmac(Lam[6], -0.43392857142857144, Ops::fmac(Lam[5], -0.2892857142857143, m10))); y[10] = Ops::fma3(k, x[14], y[10]); y[14] = Ops::fma3(k, x[10], y[14]); }
      { k = Ops::mulc(w55, -0.2892857142857143); y[10] = Ops::fma3(k, x[15], y[10]); y[15] = Ops::fma3(k, x[10], y[15]); }
      { k = Ops::fmac(w46, 1.4464285714285714, Ops::mulc(w38, 0.5785714285714286)); y[10] = Ops::fma3(k, x[16], y[10]); y[16] = Ops::fma3(k, x[10], y[16]); }
      { k = Ops::fmac(w17, -0.14464285714285716, Ops::fmac(w14, 0.5785714285714286, Ops::mulc(w12, 0.7232142857142857))); y[10] = Ops::fma3(k, x[17], y[10]); y[17] = Ops::fma3(k, x[10], y[17]); }
      { k = Ops::fmac(w31, -0.14464285714285716, Ops::fmac(w12, -0.2892857142857143, m8)); y[10] = Ops::fma3(k, x[18], y[10]); y[18] = Ops::fma3(k, x[10], y[18]); }
      { k = Ops::fmac(w51, -0.2892857142857143, Ops::mulc(w19, 0.5785714285714286)); y[10] = Ops::fma3(k, x[19], y[10]); y[19] = Ops::fma3(k, x[10], y[19]); }
      { k = Ops::fmac(w17, 1.1571428571428573, Ops::fmac(Lam[7], 1.4464285714285714, m7)); y[11] = Ops::fma3(k, x[11], y[11]); }
      { k = Ops::fmac(w18, -0.14464285714285716, Ops::fmac(Lam[8], -0.43392857142857144, Ops::fmac(Lam[5], -0.2892857142857143, m10))); y[11] = Ops::fma3(k, x[12], y[11]); y[12] = Ops::fma3(k, x[11], y[12]); }
      { k = Ops::fmac(w36, -0.14464285714285716, Ops::mulc(Lam[8], -0.2892857142857143)); y[11] = Ops::fma3(k, x[13], y[11]); y[13] = Ops::fma3(k, x[11], y[13]); }
      { k = Ops::fmac(w2, 0.5785714285714286, Ops::fmac(Lam[7], 0.7232142857142857, Ops::fmac(Lam[6], 1.1571428571428573, m9))); y[11] = Ops::fma3(k, x[14], y[11]); y[14] = Ops::fma3(k, x[11], y[14]); }
      { k = Ops::fmac(w24, -0.14464285714285716, Ops::fmac(Lam[8], -0.2892857142857143, Ops::fmac(Lam[6], -0.43392857142857144, m10))); y[11] = Ops::fma3(k, x[15], y[11]); y[15] = Ops::fma3(k, x[11], y[15]); }
      { k = Ops::fmac(w48, 1.4464285714285714, Ops::mulc(w37, 0.5785714285714286)); y[11] = Ops::fma3(k, x[16], y[11]); y[16] = Ops::fma3(k, x[11], y[16]); }
      { k = Ops::fmac(w42, -0.14464285714285716, Ops::fmac(w14, -0.2892857142857143, m8)); y[11] = Ops::fma3(k, x[17], y[11]); y[17] = Ops::fma3(k, x[11], y[17]); }
      { k = Ops::fmac(w24, -0.14464285714285716, Ops::fmac(w14, 0.7232142857142857, Ops::mulc(w12, 0.5785714285714286))); y[11] = Ops::fma3(k, x[18], y[11]); y[18] = Ops::fma3(k, x[11], y[18]); }
      { k = Ops::fmac(w56, -0.2892857142857143, Ops::mulc(w36, 0.5785714285714286)); y[11] = Ops::fma3(k, x[19], y[11]); y[19] = Ops::fma3(k, x[11], y[19]); }
      { k = Ops::fmac(w25, 1.1571428571428573, Ops::fmac(Lam[4], 1.4464285714285714, m7)); y[12] = Ops::fma3(k, x[12], y[12]); }
      { k = Ops::fmac(Lam[9], -0.43392857142857144, Ops::fmac(Lam[6], 0.2892857142857143, Ops::fmac(Lam[4], -0.43392857142857144, m8))); y[12] = Ops::fma3(k, x[13], y[12]); y[13] = Ops::fma3(k, x[12], y[13]); }
      { k = Ops::fmac(w40, -0.14464285714285716, Ops::mulc(Lam[5], -0.2892857142857143)); y[12] = Ops::fma3(k, x[14], y[12]); y[14] = Ops::fma3(k, x[12], y[14]); }
      { k = Ops::fmac(w6, -0.14464285714285716, Ops::fmac(Lam[6], -0.2892857142857143, Ops::fmac(Lam[5], -0.43392857142857144, m10))); y[12] = Ops::fma3(k, x[15], y[12]); y[15] = Ops::fma3(k, x[12], y[15]); }
      { k = Ops::fmac(w18, -0.14464285714285716, Ops::fmac(w15, 0.5785714285714286, Ops::mulc(w11, 0.7232142857142857))); y[12] = Ops::fma3(k, x[16], y[12]); y[16] = Ops::fma3(k, x[12], y[16]); }
      { k = Ops::fmac(w46, 1.4464285714285714, Ops::mulc(w20, 0.5785714285714286)); y[12] = Ops::fma3(k, x[17], y[12]); y[17] = Ops::fma3(k, x[12], y[17]); }
      { k = Ops::fmac(w29, -0.14464285714285716, Ops::fmac(w11, -0.2892857142857143, m8)); y[12] = Ops::fma3(k, x[18], y[12]); y[18] = Ops::fma3(k, x[12], y[18]); }
      { k = Ops::fmac(w50, -0.2892857142857143, Ops::mulc(w40, 0.5785714285714286)); y[12] = Ops::fma3(k, x[19], y[12]); y[19] = Ops::fma3(k, x[12], y[19]); }
      { k = Ops::fmac(w18, 1.1571428571428573, Ops::fmac(Lam[9], 1.4464285714285714, m7)); y[13] = Ops::fma3(k, x[13], y[13]); }
      { k = Ops::fmac(w25, -0.14464285714285716, Ops::fmac(Lam[8], -0.2892857142857143, Ops::fmac(Lam[5], -0.43392857142857144, m10))); y[13] = Ops::fma3(k, x[14], y[13]); y[14] = Ops::fma3(k, x[13], y[14]); }
      { k = Ops::fmac(w10, 0.5785714285714286, Ops::fmac(Lam[9], 0.7232142857142857, Ops::fmac(Lam[5], 1.1571428571428573, m9))); y[13] = Ops::fma3(k, x[15], y[13]); y[15] = Ops::fma3(k, x[13], y[15]); }
      { k = Ops::fmac(w42, -0.14464285714285716, Ops::fmac(w15, -0.2892857142857143, m8)); y[13] = Ops::fma3(k, x[16], y[13]); y[16] = Ops::fma3(k, x[13], y[16]); }
      { k = Ops::fmac(w49, 1.4464285714285714, Ops::mulc(w39, 0.5785714285714286)); y[13] = Ops::fma3(k, x[17], y[13]); y[17] = Ops::fma3(k, x[13], y[17]); }
      { k = Ops::fmac(w25, -0.14464285714285716, Ops::fmac(w15, 0.7232142857142857, Ops::mulc(w11, 0.5785714285714286))); y[13] = Ops::fma3(k, x[18], y[13]); y[18] = Ops::fma3(k, x[13], y[18]); }
      { k = Ops::fmac(w57, 1.4464285714285714, Ops::mulc(w36, 0.5785714285714286)); y[13] = Ops::fma3(k, x[19], y[13]); y[19] = Ops::fma3(k, x[13], y[19]); }
      { k = Ops::fmac(w6, 1.1571428571428573, Ops::fmac(Lam[7], 1.4464285714285714, m7)); y[14] = Ops::fma3(k, x[14], y[14]); }
      { k = Ops::fmac(Lam[9], -0.43392857142857144, Ops::fmac(Lam[8], 0.2892857142857143, Ops::fmac(Lam[7], -0.43392857142857144, m8))); y[14] = Ops::fma3(k, x[15], y[14]); y[15] = Ops::fma3(k, x[14], y[15]); }
      { k = Ops::fmac(w26, -0.14464285714285716, Ops::fmac(w9, 0.7232142857142857, Ops::mulc(w1, 0.5785714285714286))); y[14] = Ops::fma3(k, x[16], y[14]); y[16] = Ops::fma3(k, x[14], y[16]); }
      { k = Ops::fmac(w29, -0.14464285714285716, Ops::fmac(w9, -0.2892857142857143, m8)); y[14] = Ops::fma3(k, x[17], y[14]); y[17] = Ops::fma3(k, x[14], y[17]); }
      { k = Ops::fmac(w48, 1.4464285714285714, Ops::mulc(w35, 0.5785714285714286)); y[14] = Ops::fma3(k, x[18], y[14]); y[18] = Ops::fma3(k, x[14], y[18]); }
      { k = Ops::fmac(w52, 1.4464285714285714, Ops::mulc(w40, 0.5785714285714286)); y[14] = Ops::fma3(k, x[19], y[14]); y[19] = Ops::fma3(k, x[14], y[19]); }
      { k = Ops::fmac(w26, 1.1571428571428573, Ops::fmac(Lam[9], 1.4464285714285714, m7)); y[15] = Ops::fma3(k, x[15], y[15]); }
      { k = Ops::fmac(w31, -0.14464285714285716, Ops::fmac(w1, -0.2892857142857143, m8)); y[15] = Ops::fma3(k, x[16], y[15]); y[16] = Ops::fma3(k, x[15], y[16]); }
      { k = Ops::fmac(w9, 0.5785714285714286, Ops::fmac(w6, -0.14464285714285716, Ops::mulc(w1, 0.7232142857142857))); y[15] = Ops::fma3(k, x[17], y[15]); y[17] = Ops::fma3(k, x[15], y[17]); }
      { k = Ops::fmac(w49, 1.4464285714285714, Ops::mulc(w41, 0.5785714285714286)); y[15] = Ops::fma3(k, x[18], y[15]); y[18] = Ops::fma3(k, x[15], y[18]); }
      { k = Ops::fmac(w54, 1.4464285714285714, Ops::mulc(w19, 0.5785714285714286)); y[15] = Ops::fma3(k, x[19], y[15]); y[19] = Ops::fma3(k, x[15], y[19]); }
      { k = Ops::fmac(w59, 3.4714285714285715, Ops::fmac(Lam[7], 3.4714285714285715, m11)); y[16] = Ops::fma3(k, x[16], y[16]); }
      { k = Ops::fmac(w59, 1.7357142857142858, Ops::fmac(w1, 1.7357142857142858, Ops::fmac(Lam[8], 3.4714285714285715, m12))); y[16] = Ops::fma3(k, x[17], y[16]); y[17] = Ops::fma3(k, x[16], y[17]); }
      { k = Ops::fmac(w55, 3.4714285714285715, Ops::fmac(w27, 1.7357142857142858, m12)); y[16] = Ops::fma3(k, x[18], y[16]); y[18] = Ops::fma3(k, x[16], y[18]); }
      { k = Ops::fmac(w60, 1.7357142857142858, Ops::fmac(w0, 1.7357142857142858, Ops::fmac(Lam[3], 3.4714285714285715, m12))); y[16] = Ops::fma3(k, x[19], y[16]); y[19] = Ops::fma3(k, x[16], y[19]); }
      { k = Ops::fmac(w58, 3.4714285714285715, Ops::fmac(Lam[0], 3.4714285714285715, m11)); y[17] = Ops::fma3(k, x[17], y[17]); }
      { k = Ops::fmac(w53, 3.4714285714285715, Ops::fmac(w29, 1.7357142857142858, m12)); y[17] = Ops::fma3(k, x[18], y[17]); y[18] = Ops::fma3(k, x[17], y[18]); }
      { k = Ops::fmac(w58, 1.7357142857142858, Ops::fmac(w2, 1.7357142857142858, Ops::fmac(Lam[2], 3.4714285714285715, m12))); y[17] = Ops::fma3(k, x[19], y[17]); y[19] = Ops::fma3(k, x[17], y[19]); }
      { k = Ops::fmac(w6, 3.4714285714285715, Ops::fmac(w5, 3.4714285714285715, Ops::fmac(w3, 3.4714285714285715, m11))); y[18] = Ops::fma3(k, x[18], y[18]); }
      { k = Ops::fmac(w47, 3.4714285714285715, Ops::fmac(w31, 1.7357142857142858, m12)); y[18] = Ops::fma3(k, x[19], y[18]); y[19] = Ops::fma3(k, x[18], y[19]); }
      { k = Ops::fmac(w60, 3.4714285714285715, Ops::fmac(Lam[9], 3.4714285714285715, m11)); y[19] = Ops::fma3(k, x[19], y[19]); }
    }
    else if constexpr (STIFF) {
      const typename Ops::T w0 = Ops::add(Lam[1], Lam[2]);
      const typename Ops::T w1 = Ops::add(Lam[3], Lam[6]);
      const typename Ops::T w2 = Ops::add(Lam[5], Lam[8]);
      const typename Ops::T w3 = Ops::add(Lam[0], Lam[3]);
      const typename Ops::T w4 = Ops::add(Lam[1], Lam[4]);
      const typename Ops::T w5 = Ops::add(Lam[2], Lam[7]);
      const typename Ops::T w6 = Ops::add(Lam[8], Lam[9]);
      const typename Ops::T w7 = Ops::add(Lam[5], Lam[6]);
      const typename Ops::T w8 = Ops::add(Lam[1], Lam[3]);
      const typename Ops::T w9 = Ops::add(Lam[2], Lam[5]);
      const typename Ops::T w10 = Ops::add(Lam[6], Lam[8]);
      const typename Ops::T w11 = Ops::add(Lam[1], Lam[5]);
      const typename Ops::T w12 = Ops::add(Lam[1], Lam[6]);
      const typename Ops::T w13 = Ops::add(Lam[2], Lam[3]);
      const typename Ops::T w14 = Ops::add(Lam[2], Lam[8]);
      const typename Ops::T w15 = Ops::add(Lam[3], Lam[8]);
      const typename Ops::T w16 = Ops::add(Lam[0], w0);
      const typename Ops::T w17 = Ops::add(Lam[4], Lam[5]);
      const typename Ops::T w18 = Ops::add(Lam[4], Lam[6]);
      const typename Ops::T w19 = Ops::add(Lam[7], w2);
      const typename Ops::T w20 = Ops::add(Lam[9], w1);
      const typename Ops::T w21 = Ops::add(Lam[0], Lam[1]);
      const typename Ops::T w22 = Ops::add(Lam[0], Lam[2]);
      const typename Ops::T w23 = Ops::add(Lam[3], Lam[9]);
      const typename Ops::T w24 = Ops::add(Lam[5], Lam[7]);
      const typename Ops::T w25 = Ops::add(Lam[6], Lam[9]);
      const typename Ops::T w26 = Ops::add(Lam[7], Lam[8]);
      const typename Ops::T w27 = Ops::add(w0, w3);
      const typename Ops::T w28 = Ops::add(w0, w10);
      const typename Ops::T w29 = Ops::add(w1, w6);
      const typename Ops::T w30 = Ops::add(w1, w9);
      const typename Ops::T w31 = Ops::add(w2, w5);
      const typename Ops::T w32 = Ops::add(w2, w8);
      const typename Ops::T w33 = Ops::add(Lam[1], w3);
      const typename Ops::T w34 = Ops::add(Lam[2], w3);
      const typename Ops::T w35 = Ops::add(Lam[3], w6);
      const typename Ops::T w36 = Ops::add(Lam[4], w7);
      const typename Ops::T w37 = Ops::add(Lam[5], w4);
      const typename Ops::T w38 = Ops::add(Lam[5], w5);
      const typename Ops::T w39 = Ops::add(Lam[6], w4);
      const typename Ops::T w40 = Ops::add(Lam[6], w6);
      const typename Ops::T w41 = Ops::add(Lam[8], w5);
      const typename Ops::T w42 = Ops::add(w4, w7);
      const typename Ops::T w43 = Ops::fmac(Lam[1], -5.0, Lam[0]);
      const typename Ops::T w44 = Ops::fmac(Lam[2], -5.0, Lam[0]);
      const typename Ops::T w45 = Ops::fmac(Lam[3], -5.0, Lam[0]);
      const typename Ops::T w46 = Ops::fmac(Lam[4], -0.2, Lam[1]);
      const typename Ops::T w47 = Ops::fmac(w20, 0.5, Lam[1]);
      const typename Ops::T w48 = Ops::fmac(Lam[7], -0.2, Lam[2]);
      const typename Ops::T w49 = Ops::fmac(Lam[9], -0.2, Lam[3]);
      const typename Ops::T w50 = Ops::fmac(Lam[5], -5.0, Lam[4]);
      const typename Ops::T w51 = Ops::fmac(Lam[6], -5.0, Lam[4]);
      const typename Ops::T w52 = Ops::fmac(Lam[7], -0.2, Lam[5]);
      const typename Ops::T w53 = Ops::fmac(w16, 0.5, Lam[5]);
      const typename Ops::T w54 = Ops::fmac(Lam[9], -0.2, Lam[6]);
      const typename Ops::T w55 = Ops::fmac(w19, 0.5, Lam[6]);
      const typename Ops::T w56 = Ops::fmac(Lam[8], -5.0, Lam[7]);
      const typename Ops::T w57 = Ops::fmac(Lam[9], -0.2, Lam[8]);
      const typename Ops::T w58 = Ops::add(w4, w20);
      const typename Ops::T w59 = Ops::add(w16, w17);
      const typename Ops::T w60 = Ops::add(w18, w19);
      { k = Ops::mulc(Lam[0], 0.35714285714285715); y[0] = Ops::mul(k, x[0]); }
      { k = Ops::mulc(Lam[1], 0.06785714285714285); y[0] = Ops::fma3(k, x[1], y[0]); y[1] = Ops::mul(k, x[0]); }
      { k = Ops::mulc(Lam[2], 0.06785714285714285); y[0] = Ops::fma3(k, x[2], y[0]); y[2] = Ops::mul(k, x[0]); }
      { k = Ops::mulc(Lam[3], 0.06785714285714285); y[0] = Ops::fma3(k, x[3], y[0]); y[3] = Ops::mul(k, x[0]); }
      { k = Ops::fmac(Lam[1], 0.36964285714285716, Ops::mulc(Lam[0], -0.20892857142857144)); y[0] = Ops::fma3(k, x[4], y[0]); y[4] = Ops::mul(k, x[0]); }
      { k = Ops::fmac(Lam[1], -0.20892857142857144, Ops::mulc(Lam[0], 0.08035714285714286)); y[0] = Ops::fma3(k, x[5], y[0]); y[5] = Ops::mul(k, x[0]); }
      { k = Ops::fmac(Lam[2], 0.36964285714285716, Ops::mulc(Lam[0], -0.20892857142857144)); y[0] = Ops::fma3(k, x[6], y[0]); y[6] = Ops::mul(k, x[0]); }
      { k = Ops::fmac(Lam[2], -0.20892857142857144, Ops::mulc(Lam[0], 0.08035714285714286)); y[0] = Ops::fma3(k, x[7], y[0]); y[7] = Ops::mul(k, x[0]); }
      { k = Ops::fmac(Lam[3], 0.36964285714285716, Ops::mulc(Lam[0], -0.20892857142857144)); y[0] = Ops::fma3(k, x[8], y[0]); y[8] = Ops::mul(k, x[0]); }
      { k = Ops::fmac(Lam[3], -0.20892857142857144, Ops::mulc(Lam[0], 0.08035714285714286)); y[0] = Ops::fma3(k, x[9], y[0]); y[9] = Ops::mul(k, x[0]); }
      { k = Ops::mulc(w0, 0.08035714285714286); y[0] = Ops::fma3(k, x[10], y[0]); y[10] = Ops::mul(k, x[0]); }
      { k = Ops::mulc(w0, 0.08035714285714286); y[0] = Ops::fma3(k, x[11], y[0]); y[11] = Ops::mul(k, x[0]); }
      { k = Ops::mulc(w8, 0.08035714285714286); y[0] = Ops::fma3(k, x[12], y[0]); y[12] = Ops::mul(k, x[0]); }
      { k = Ops::mulc(w8, 0.08035714285714286); y[0] = Ops::fma3(k, x[13], y[0]); y[13] = Ops::mul(k, x[0]); }
      { k = Ops::mulc(w13, 0.08035714285714286); y[0] = Ops::fma3(k, x[14], y[0]); y[14] = Ops::mul(k, x[0]); }
      { k = Ops::mulc(w13, 0.08035714285714286); y[0] = Ops::fma3(k, x[15], y[0]); y[15] = Ops::mul(k, x[0]); }
      { k = Ops::fmac(w0, -0.09642857142857143, Ops::mulc(Lam[0], 0.19285714285714287)); y[0] = Ops::fma3(k, x[16], y[0]); y[16] = Ops::mul(k, x[0]); }
      { k = Ops::fmac(w8, -0.09642857142857143, Ops::mulc(Lam[0], 0.19285714285714287)); y[0] = Ops::fma3(k, x[17], y[0]); y[17] = Ops::mul(k, x[0]); }
      { k = Ops::fmac(w13, -0.09642857142857143, Ops::mulc(Lam[0], 0.19285714285714287)); y[0] = Ops::fma3(k, x[18], y[0]); y[18] = Ops::mul(k, x[0]); }
      { k = Ops::fmac(w0, 0.19285714285714287, Ops::mulc(Lam[3], 0.19285714285714287)); y[0] = Ops::fma3(k, x[19], y[0]); y[19] = Ops::mul(k, x[0]); }
      { k = Ops::mulc(Lam[4], 0.35714285714285715); y[1] = Ops::fma3(k, x[1], y[1]); }
      { k = Ops::mulc(Lam[5], 0.06785714285714285); y[1] = Ops::fma3(k, x[2], y[1]); y[2] = Ops::fma3(k, x[1], y[2]); }
      { k = Ops::mulc(Lam[6], 0.06785714285714285); y[1] = Ops::fma3(k, x[3], y[1]); y[3] = Ops::fma3(k, x[1], y[3]); }
      { k = Ops::fmac(Lam[4], 0.08035714285714286, Ops::mulc(Lam[1], -0.20892857142857144)); y[1] = Ops::fma3(k, x[4], y[1]); y[4] = Ops::fma3(k, x[1], y[4]); }
      { k = Ops::fmac(Lam[4], -0.20892857142857144, Ops::mulc(Lam[1], 0.36964285714285716)); y[1] = Ops::fma3(k, x[5], y[1]); y[5] = Ops::fma3(k, x[1], y[5]); }
      { k = Ops::mulc(w11, 0.08035714285714286); y[1] = Ops::fma3(k, x[6], y[1]); y[6] = Ops::fma3(k, x[1], y[6]); }
      { k = Ops::mulc(w11, 0.08035714285714286); y[1] = Ops::fma3(k, x[7], y[1]); y[7] = Ops::fma3(k, x[1], y[7]); }
      { k = Ops::mulc(w12, 0.08035714285714286); y[1] = Ops::fma3(k, x[8], y[1]); y[8] = Ops::fma3(k, x[1], y[8]); }
      { k = Ops::mulc(w12, 0.08035714285714286); y[1] = Ops::fma3(k, x[9], y[1]); y[9] = Ops::fma3(k, x[1], y[9]); }
      { k = Ops::fmac(Lam[5], 0.36964285714285716, Ops::mulc(Lam[4], -0.20892857142857144)); y[1] = Ops::fma3(k, x[10], y[1]); y[10] = Ops::fma3(k, x[1], y[10]); }
      { k = Ops::fmac(Lam[5], -0.20892857142857144, Ops::mulc(Lam[4], 0.08035714285714286)); y[1] = Ops::fma3(k, x[11], y[1]); y[11] = Ops::fma3(k, x[1], y[11]); }
      { k = Ops::fmac(Lam[6], 0.36964285714285716, Ops::mulc(Lam[4], -0.20892857142857144)); y[1] = Ops::fma3(k, x[12], y[1]); y[12] = Ops::fma3(k, x[1], y[12]); }
      { k = Ops::fmac(Lam[6], -0.20892857142857144, Ops::mulc(Lam[4], 0.08035714285714286)); y[1] = Ops::fma3(k, x[13], y[1]); y[13] = Ops::fma3(k, x[1], y[13]); }
      { k = Ops::mulc(w7, 0.08035714285714286); y[1] = Ops::fma3(k, x[14], y[1]); y[14] = Ops::fma3(k, x[1], y[14]); }
      { k = Ops::mulc(w7, 0.08035714285714286); y[1] = Ops::fma3(k, x[15], y[1]); y[15] = Ops::fma3(k, x[1], y[15]); }
      { k = Ops::fmac(w11, -0.09642857142857143, Ops::mulc(Lam[4], 0.19285714285714287)); y[1] = Ops::fma3(k, x[16], y[1]); y[16] = Ops::fma3(k, x[1], y[16]); }
      { k = Ops::fmac(w12, -0.09642857142857143, Ops::mulc(Lam[4], 0.19285714285714287)); y[1] = Ops::fma3(k, x[17], y[1]); y[17] = Ops::fma3(k, x[1], y[17]); }
      { k = Ops::fmac(w7, 0.19285714285714287, Ops::mulc(Lam[1], 0.19285714285714287)); y[1] = Ops::fma3(k, x[18], y[1]); y[18] = Ops::fma3(k, x[1], y[18]); }
      { k = Ops::fmac(w7, -0.09642857142857143, Ops::mulc(Lam[4], 0.19285714285714287)); y[1] = Ops::fma3(k, x[19], y[1]); y[19] = Ops::fma3(k, x[1], y[19]); }
      { k = Ops::mulc(Lam[7], 0.35714285714285715); y[2] = Ops::fma3(k, x[2], y[2]); }
      { k = Ops::mulc(Lam[8], 0.06785714285714285); y[2] = Ops::fma3(k, x[3], y[2]); y[3] = Ops::fma3(k, x[2], y[3]); }
      { k = Ops::mulc(w9, 0.08035714285714286); y[2] = Ops::fma3(k, x[4], y[2]); y[4] = Ops::fma3(k, x[2], y[4]); }
      { k = Ops::mulc(w9, 0.08035714285714286); y[2] = Ops::fma3(k, x[5], y[2]); y[5] = Ops::fma3(k, x[2], y[5]); }
      { k = Ops::fmac(Lam[7], 0.08035714285714286, Ops::mulc(Lam[2], -0.20892857142857144)); y[2] = Ops::fma3(k, x[6], y[2]); y[6] = Ops::fma3(k, x[2], y[6]); }
      { k = Ops::fmac(Lam[7], -0.20892857142857144, Ops::mulc(Lam[2], 0.36964285714285716)); y[2] = Ops::fma3(k, x[7], y[2]); y[7] = Ops::fma3(k, x[2], y[7]); }
      { k = Ops::mulc(w14, 0.08035714285714286); y[2] = Ops::fma3(k, x[8], y[2]); y[8] = Ops::fma3(k, x[2], y[8]); }
      { k = Ops::mulc(w14, 0.08035714285714286); y[2] = Ops::fma3(k, x[9], y[2]); y[9] = Ops::fma3(k, x[2], y[9]); }
      { k = Ops::fmac(Lam[7], 0.08035714285714286, Ops::mulc(Lam[5], -0.20892857142857144)); y[2] = Ops::fma3(k, x[10], y[2]); y[10] = Ops::fma3(k, x[2], y[10]); }
      { k = Ops::fmac(Lam[7], -0.20892857142857144, Ops::mulc(Lam[5], 0.36964285714285716)); y[2] = Ops::fma3(k, x[11], y[2]); y[11] = Ops::fma3(k, x[2], y[11]); }
      { k = Ops::mulc(w2, 0.08035714285714286); y[2] = Ops::fma3(k, x[12], y[2]); y[12] = Ops::fma3(k, x[2], y[12]); }
      { k = Ops::mulc(w2, 0.08035714285714286); y[2] = Ops::fma3(k, x[13], y[2]); y[13] = Ops::fma3(k, x[2], y[13]); }
      { k = Ops::fmac(Lam[8], 0.36964285714285716, Ops::mulc(Lam[7], -0.20892857142857144)); y[2] = Ops::fma3(k, x[14], y[2]); y[14] = Ops::fma3(k, x[2], y[14]); }
      { k = Ops::fmac(Lam[8], -0.20892857142857144, Ops::mulc(Lam[7], 0.08035714285714286)); y[2] = Ops::fma3(k, x[15], y[2]); y[15] = Ops::fma3(k, x[2], y[15]); }
      { k = Ops::fmac(w9, -0.09642857142857143, Ops::mulc(Lam[7], 0.19285714285714287)); y[2] = Ops::fma3(k, x[16], y[2]); y[16] = Ops::fma3(k, x[2], y[16]); }
      { k = Ops::fmac(w2, 0.19285714285714287, Ops::mulc(Lam[2], 0.19285714285714287)); y[2] = Ops::fma3(k, x[17], y[2]); y[17] = Ops::fma3(k, x[2], y[17]); }
      { k = Ops::fmac(w14, -0.09642857142857143, Ops::mulc(Lam[7], 0.19285714285714287)); y[2] = Ops::fma3(k, x[18], y[2]); y[18] = Ops::fma3(k, x[2], y[18]); }
      { k = Ops::fmac(w2, -0.09642857142857143, Ops::mulc(Lam[7], 0.19285714285714287)); y[2] = Ops::fma3(k, x[19], y[2]); y[19] = Ops::fma3(k, x[2], y[19]); }
      { k = Ops::mulc(Lam[9], 0.35714285714285715); y[3] = Ops::fma3(k, x[3], y[3]); }
      { k = Ops::mulc(w1, 0.08035714285714286); y[3] = Ops::fma3(k, x[4], y[3]); y[4] = Ops::fma3(k, x[3], y[4]); }
      { k = Ops::mulc(w1, 0.08035714285714286); y[3] = Ops::fma3(k, x[5], y[3]); y[5] = Ops::fma3(k, x[3], y[5]); }
      { k = Ops::mulc(w15, 0.08035714285714286); y[3] = Ops::fma3(k, x[6], y[3]); y[6] = Ops::fma3(k, x[3], y[6]); }
      { k = Ops::mulc(w15, 0.08035714285714286); y[3] = Ops::fma3(k, x[7], y[3]); y[7] = Ops::fma3(k, x[3], y[7]); }
      { k = Ops::fmac(Lam[9], 0.08035714285714286, Ops::mulc(Lam[3], -0.20892857142857144)); y[3] = Ops::fma3(k, x[8], y[3]); y[8] = Ops::fma3(k, x[3], y[8]); }
      { k = Ops::fmac(Lam[9], -0.20892857142857144, Ops::mulc(Lam[3], 0.36964285714285716)); y[3] = Ops::fma3(k, x[9], y[3]); y[9] = Ops::fma3(k, x[3], y[9]); }
      { k = Ops::mulc(w10, 0.08035714285714286); y[3] = Ops::fma3(k, x[10], y[3]); y[10] = Ops::fma3(k, x[3], y[10]); }
      { k = Ops::mulc(w10, 0.08035714285714286); y[3] = Ops::fma3(k, x[11], y[3]); y[11] = Ops::fma3(k, x[3], y[11]); }
      { k = Ops::fmac(Lam[9], 0.08035714285714286, Ops::mulc(Lam[6], -0.20892857142857144)); y[3] = Ops::fma3(k, x[12], y[3]); y[12] = Ops::fma3(k, x[3], y[12]); }
      { k = Ops::fmac(Lam[9], -0.20892857142857144, Ops::mulc(Lam[6], 0.36964285714285716)); y[3] = Ops::fma3(k, x[13], y[3]); y[13] = Ops::fma3(k, x[3], y[13]); }
      { k = Ops::fmac(Lam[9], 0.08035714285714286, Ops::mulc(Lam[8], -0.20892857142857144)); y[3] = Ops::fma3(k, x[14], y[3]); y[14] = Ops::fma3(k, x[3], y[14]); }
      { k = Ops::fmac(Lam[9], -0.20892857142857144, Ops::mulc(Lam[8], 0.36964285714285716)); y[3] = Ops::fma3(k, x[15], y[3]); y[15] = Ops::fma3(k, x[3], y[15]); }
      { k = Ops::fmac(w1, 0.19285714285714287, Ops::mulc(Lam[8], 0.19285714285714287)); y[3] = Ops::fma3(k, x[16], y[3]); y[16] = Ops::fma3(k, x[3], y[16]); }
      { k = Ops::fmac(w1, -0.09642857142857143, Ops::mulc(Lam[9], 0.19285714285714287)); y[3] = Ops::fma3(k, x[17], y[3]); y[17] = Ops::fma3(k, x[3], y[17]); }
      { k = Ops::fmac(w15, -0.09642857142857143, Ops::mulc(Lam[9], 0.19285714285714287)); y[3] = Ops::fma3(k, x[18], y[3]); y[18] = Ops::fma3(k, x[3], y[18]); }
      { k = Ops::fmac(w10, -0.09642857142857143, Ops::mulc(Lam[9], 0.19285714285714287)); y[3] = Ops::fma3(k, x[19], y[3]); y[19] = Ops::fma3(k, x[3], y[19]); }
      { k = Ops::fmac(w4, 1.1571428571428573, Ops::mulc(Lam[0], 1.4464285714285714)); y[4] = Ops::fma3(k, x[4], y[4]); }
      { k = Ops::fmac(Lam[4], -0.43392857142857144, Ops::fmac(Lam[1], 0.2892857142857143, Ops::mulc(Lam[0], -0.43392857142857144))); y[4] = Ops::fma3(k, x[5], y[4]); y[5] = Ops::fma3(k, x[4], y[5]); }
      { k = Ops::fmac(w0, 0.5785714285714286, Ops::fmac(Lam[5], 1.1571428571428573, Ops::mulc(Lam[0], 0.7232142857142857))); y[4] = Ops::fma3(k, x[6], y[4]); y[6] = Ops::fma3(k, x[4], y[6]); }
      { k = Ops::fmac(w21, -0.14464285714285716, Ops::fmac(Lam[5], -0.43392857142857144, Ops::mulc(Lam[2], -0.2892857142857143))); y[4] = Ops::fma3(k, x[7], y[4]); y[7] = Ops::fma3(k, x[4], y[7]); }
      { k = Ops::fmac(w8, 0.5785714285714286, Ops::fmac(Lam[6], 1.1571428571428573, Ops::mulc(Lam[0], 0.7232142857142857))); y[4] = Ops::fma3(k, x[8], y[4]); y[8] = Ops::fma3(k, x[4], y[8]); }
      { k = Ops::fmac(w21, -0.14464285714285716, Ops::fmac(Lam[6], -0.43392857142857144, Ops::mulc(Lam[3], -0.2892857142857143))); y[4] = Ops::fma3(k, x[9], y[4]); y[9] = Ops::fma3(k, x[4], y[9]); }
      { k = Ops::fmac(w17, -0.14464285714285716, Ops::fmac(Lam[2], -0.43392857142857144, Ops::mulc(Lam[1], -0.2892857142857143))); y[4] = Ops::fma3(k, x[10], y[4]); y[10] = Ops::fma3(k, x[4], y[10]); }
      { k = Ops::fmac(w37, -0.14464285714285716, Ops::mulc(Lam[2], -0.2892857142857143)); y[4] = Ops::fma3(k, x[11], y[4]); y[11] = Ops::fma3(k, x[4], y[11]); }
      { k = Ops::fmac(w18, -0.14464285714285716, Ops::fmac(Lam[3], -0.43392857142857144, Ops::mulc(Lam[1], -0.2892857142857143))); y[4] = Ops::fma3(k, x[12], y[4]); y[12] = Ops::fma3(k, x[4], y[12]); }
      { k = Ops::fmac(w39, -0.14464285714285716, Ops::mulc(Lam[3], -0.2892857142857143)); y[4] = Ops::fma3(k, x[13], y[4]); y[13] = Ops::fma3(k, x[4], y[13]); }
      { k = Ops::mulc(w30, -0.14464285714285716); y[4] = Ops::fma3(k, x[14], y[4]); y[14] = Ops::fma3(k, x[4], y[14]); }
      { k = Ops::mulc(w30, -0.14464285714285716); y[4] = Ops::fma3(k, x[15], y[4]); y[15] = Ops::fma3(k, x[4], y[15]); }
      { k = Ops::fmac(w44, -0.2892857142857143, Ops::mulc(w37, 0.5785714285714286)); y[4] = Ops::fma3(k, x[16], y[4]); y[16] = Ops::fma3(k, x[4], y[16]); }
      { k = Ops::fmac(w45, -0.2892857142857143, Ops::mulc(w39, 0.5785714285714286)); y[4] = Ops::fma3(k, x[17], y[4]); y[17] = Ops::fma3(k, x[4], y[17]); }
      { k = Ops::fmac(w21, -0.14464285714285716, Ops::fmac(w13, 0.7232142857142857, Ops::mulc(w7, 0.5785714285714286))); y[4] = Ops::fma3(k, x[18], y[4]); y[18] = Ops::fma3(k, x[4], y[18]); }
      { k = Ops::fmac(w42, -0.14464285714285716, Ops::mulc(w13, -0.2892857142857143)); y[4] = Ops::fma3(k, x[19], y[4]); y[19] = Ops::fma3(k, x[4], y[19]); }
      { k = Ops::fmac(w21, 1.1571428571428573, Ops::mulc(Lam[4], 1.4464285714285714)); y[5] = Ops::fma3(k, x[5], y[5]); }
      { k = Ops::fmac(w22, -0.14464285714285716, Ops::fmac(Lam[5], -0.43392857142857144, Ops::mulc(Lam[1], -0.2892857142857143))); y[5] = Ops::fma3(k, x[6], y[5]); y[6] = Ops::fma3(k, x[5], y[6]); }
      { k = Ops::mulc(w53, -0.2892857142857143); y[5] = Ops::fma3(k, x[7], y[5]); y[7] = Ops::fma3(k, x[5], y[7]); }
      { k = Ops::fmac(w3, -0.14464285714285716, Ops::fmac(Lam[6], -0.43392857142857144, Ops::mulc(Lam[1], -0.2892857142857143))); y[5] = Ops::fma3(k, x[8], y[5]); y[8] = Ops::fma3(k, x[5], y[8]); }
      { k = Ops::fmac(w33, -0.14464285714285716, Ops::mulc(Lam[6], -0.2892857142857143)); y[5] = Ops::fma3(k, x[9], y[5]); y[9] = Ops::fma3(k, x[5], y[9]); }
      { k = Ops::fmac(w11, 0.5785714285714286, Ops::fmac(Lam[4], 0.7232142857142857, Ops::mulc(Lam[2], 1.1571428571428573))); y[5] = Ops::fma3(k, x[10], y[5]); y[10] = Ops::fma3(k, x[5], y[10]); }
      { k = Ops::fmac(w4, -0.14464285714285716, Ops::fmac(Lam[5], -0.2892857142857143, Ops::mulc(Lam[2], -0.43392857142857144))); y[5] = Ops::fma3(k, x[11], y[5]); y[11] = Ops::fma3(k, x[5], y[11]); }
      { k = Ops::fmac(w12, 0.5785714285714286, Ops::fmac(Lam[4], 0.7232142857142857, Ops::mulc(Lam[3], 1.1571428571428573))); y[5] = Ops::fma3(k, x[12], y[5]); y[12] = Ops::fma3(k, x[5], y[12]); }
      { k = Ops::fmac(w4, -0.14464285714285716, Ops::fmac(Lam[6], -0.2892857142857143, Ops::mulc(Lam[3], -0.43392857142857144))); y[5] = Ops::fma3(k, x[13], y[5]); y[13] = Ops::fma3(k, x[5], y[13]); }
      { k = Ops::mulc(w30, -0.14464285714285716); y[5] = Ops::fma3(k, x[14], y[5]); y[14] = Ops::fma3(k, x[5], y[14]); }
      { k = Ops::mulc(w30, -0.14464285714285716); y[5] = Ops::fma3(k, x[15], y[5]); y[15] = Ops::fma3(k, x[5], y[15]); }
      { k = Ops::fmac(w50, -0.2892857142857143, Ops::mulc(w16, 0.5785714285714286)); y[5] = Ops::fma3(k, x[16], y[5]); y[16] = Ops::fma3(k, x[5], y[16]); }
      { k = Ops::fmac(w51, -0.2892857142857143, Ops::mulc(w33, 0.5785714285714286)); y[5] = Ops::fma3(k, x[17], y[5]); y[17] = Ops::fma3(k, x[5], y[17]); }
      { k = Ops::fmac(w27, -0.14464285714285716, Ops::mulc(w7, -0.2892857142857143)); y[5] = Ops::fma3(k, x[18], y[5]); y[18] = Ops::fma3(k, x[5], y[18]); }
      { k = Ops::fmac(w13, 0.5785714285714286, Ops::fmac(w7, 0.7232142857142857, Ops::mulc(w4, -0.14464285714285716))); y[5] = Ops::fma3(k, x[19], y[5]); y[19] = Ops::fma3(k, x[5], y[19]); }
      { k = Ops::fmac(w5, 1.1571428571428573, Ops::mulc(Lam[0], 1.4464285714285714)); y[6] = Ops::fma3(k, x[6], y[6]); }
      { k = Ops::fmac(Lam[7], -0.43392857142857144, Ops::fmac(Lam[2], 0.2892857142857143, Ops::mulc(Lam[0], -0.43392857142857144))); y[6] = Ops::fma3(k, x[7], y[6]); y[7] = Ops::fma3(k, x[6], y[7]); }
      { k = Ops::fmac(w13, 0.5785714285714286, Ops::fmac(Lam[8], 1.1571428571428573, Ops::mulc(Lam[0], 0.7232142857142857))); y[6] = Ops::fma3(k, x[8], y[6]); y[8] = Ops::fma3(k, x[6], y[8]); }
      { k = Ops::fmac(w22, -0.14464285714285716, Ops::fmac(Lam[8], -0.43392857142857144, Ops::mulc(Lam[3], -0.2892857142857143))); y[6] = Ops::fma3(k, x[9], y[6]); y[9] = Ops::fma3(k, x[6], y[9]); }
      { k = Ops::fmac(w38, -0.14464285714285716, Ops::mulc(Lam[1], -0.2892857142857143)); y[6] = Ops::fma3(k, x[10], y[6]); y[10] = Ops::fma3(k, x[6], y[10]); }
      { k = Ops::fmac(w24, -0.14464285714285716, Ops::fmac(Lam[2], -0.2892857142857143, Ops::mulc(Lam[1], -0.43392857142857144))); y[6] = Ops::fma3(k, x[11], y[6]); y[11] = Ops::fma3(k, x[6], y[11]); }
      { k = Ops::mulc(w32, -0.14464285714285716); y[6] = Ops::fma3(k, x[12], y[6]); y[12] = Ops::fma3(k, x[6], y[12]); }
      { k = Ops::mulc(w32, -0.14464285714285716); y[6] = Ops::fma3(k, x[13], y[6]); y[13] = Ops::fma3(k, x[6], y[13]); }
      { k = Ops::fmac(w26, -0.14464285714285716, Ops::fmac(Lam[3], -0.43392857142857144, Ops::mulc(Lam[2], -0.2892857142857143))); y[6] = Ops::fma3(k, x[14], y[6]); y[14] = Ops::fma3(k, x[6], y[14]); }
      { k = Ops::fmac(w41, -0.14464285714285716, Ops::mulc(Lam[3], -0.2892857142857143)); y[6] = Ops::fma3(k, x[15], y[6]); y[15] = Ops::fma3(k, x[6], y[15]); }
      { k = Ops::fmac(w43, -0.2892857142857143, Ops::mulc(w38, 0.5785714285714286)); y[6] = Ops::fma3(k, x[16], y[6]); y[16] = Ops::fma3(k, x[6], y[16]); }
      { k = Ops::fmac(w22, -0.14464285714285716, Ops::fmac(w8, 0.7232142857142857, Ops::mulc(w2, 0.5785714285714286))); y[6] = Ops::fma3(k, x[17], y[6]); y[17] = Ops::fma3(k, x[6], y[17]); }
      { k = Ops::fmac(w45, -0.2892857142857143, Ops::mulc(w41, 0.5785714285714286)); y[6] = Ops::fma3(k, x[18], y[6]); y[18] = Ops::fma3(k, x[6], y[18]); }
      { k = Ops::fmac(w31, -0.14464285714285716, Ops::mulc(w8, -0.2892857142857143)); y[6] = Ops::fma3(k, x[19], y[6]); y[19] = Ops::fma3(k, x[6], y[19]); }
      { k = Ops::fmac(w22, 1.1571428571428573, Ops::mulc(Lam[7], 1.4464285714285714)); y[7] = Ops::fma3(k, x[7], y[7]); }
      { k = Ops::fmac(w3, -0.14464285714285716, Ops::fmac(Lam[8], -0.43392857142857144, Ops::mulc(Lam[2], -0.2892857142857143))); y[7] = Ops::fma3(k, x[8], y[7]); y[8] = Ops::fma3(k, x[7], y[8]); }
      { k = Ops::fmac(w34, -0.14464285714285716, Ops::mulc(Lam[8], -0.2892857142857143)); y[7] = Ops::fma3(k, x[9], y[7]); y[9] = Ops::fma3(k, x[7], y[9]); }
      { k = Ops::fmac(w5, -0.14464285714285716, Ops::fmac(Lam[5], -0.2892857142857143, Ops::mulc(Lam[1], -0.43392857142857144))); y[7] = Ops::fma3(k, x[10], y[7]); y[10] = Ops::fma3(k, x[7], y[10]); }
      { k = Ops::fmac(w9, 0.5785714285714286, Ops::fmac(Lam[7], 0.7232142857142857, Ops::mulc(Lam[1], 1.1571428571428573))); y[7] = Ops::fma3(k, x[11], y[7]); y[11] = Ops::fma3(k, x[7], y[11]); }
      { k = Ops::mulc(w32, -0.14464285714285716); y[7] = Ops::fma3(k, x[12], y[7]); y[12] = Ops::fma3(k, x[7], y[12]); }
      { k = Ops::mulc(w32, -0.14464285714285716); y[7] = Ops::fma3(k, x[13], y[7]); y[13] = Ops::fma3(k, x[7], y[13]); }
      { k = Ops::fmac(w14, 0.5785714285714286, Ops::fmac(Lam[7], 0.7232142857142857, Ops::mulc(Lam[3], 1.1571428571428573))); y[7] = Ops::fma3(k, x[14], y[7]); y[14] = Ops::fma3(k, x[7], y[14]); }
      { k = Ops::fmac(w5, -0.14464285714285716, Ops::fmac(Lam[8], -0.2892857142857143, Ops::mulc(Lam[3], -0.43392857142857144))); y[7] = Ops::fma3(k, x[15], y[7]); y[15] = Ops::fma3(k, x[7], y[15]); }
      { k = Ops::fmac(w52, 1.4464285714285714, Ops::mulc(w16, 0.5785714285714286)); y[7] = Ops::fma3(k, x[16], y[7]); y[16] = Ops::fma3(k, x[7], y[16]); }
      { k = Ops::fmac(w27, -0.14464285714285716, Ops::mulc(w2, -0.2892857142857143)); y[7] = Ops::fma3(k, x[17], y[7]); y[17] = Ops::fma3(k, x[7], y[17]); }
      { k = Ops::fmac(w56, -0.2892857142857143, Ops::mulc(w34, 0.5785714285714286)); y[7] = Ops::fma3(k, x[18], y[7]); y[18] = Ops::fma3(k, x[7], y[18]); }
      { k = Ops::fmac(w8, 0.5785714285714286, Ops::fmac(w5, -0.14464285714285716, Ops::mulc(w2, 0.7232142857142857))); y[7] = Ops::fma3(k, x[19], y[7]); y[19] = Ops::fma3(k, x[7], y[19]); }
      { k = Ops::fmac(w23, 1.1571428571428573, Ops::mulc(Lam[0], 1.4464285714285714)); y[8] = Ops::fma3(k, x[8], y[8]); }
      { k = Ops::fmac(Lam[9], -0.43392857142857144, Ops::fmac(Lam[3], 0.2892857142857143, Ops::mulc(Lam[0], -0.43392857142857144))); y[8] = Ops::fma3(k, x[9], y[8]); y[9] = Ops::fma3(k, x[8], y[9]); }
      { k = Ops::mulc(w28, -0.14464285714285716); y[8] = Ops::fma3(k, x[10], y[8]); y[10] = Ops::fma3(k, x[8], y[10]); }
      { k = Ops::mulc(w28, -0.14464285714285716); y[8] = Ops::fma3(k, x[11], y[8]); y[11] = Ops::fma3(k, x[8], y[11]); }
      { k = Ops::mulc(w47, -0.2892857142857143); y[8] = Ops::fma3(k, x[12], y[8]); y[12] = Ops::fma3(k, x[8], y[12]); }
      { k = Ops::fmac(w25, -0.14464285714285716, Ops::fmac(Lam[3], -0.2892857142857143, Ops::mulc(Lam[1], -0.43392857142857144))); y[8] = Ops::fma3(k, x[13], y[8]); y[13] = Ops::fma3(k, x[8], y[13]); }
      { k = Ops::fmac(w35, -0.14464285714285716, Ops::mulc(Lam[2], -0.2892857142857143)); y[8] = Ops::fma3(k, x[14], y[8]); y[14] = Ops::fma3(k, x[8], y[14]); }
      { k = Ops::fmac(w6, -0.14464285714285716, Ops::fmac(Lam[3], -0.2892857142857143, Ops::mulc(Lam[2], -0.43392857142857144))); y[8] = Ops::fma3(k, x[15], y[8]); y[15] = Ops::fma3(k, x[8], y[15]); }
      { k = Ops::fmac(w10, 0.5785714285714286, Ops::fmac(w3, -0.14464285714285716, Ops::mulc(w0, 0.7232142857142857))); y[8] = Ops::fma3(k, x[16], y[8]); y[16] = Ops::fma3(k, x[8], y[16]); }
      { k = Ops::fmac(w43, -0.2892857142857143, Ops::mulc(w20, 0.5785714285714286)); y[8] = Ops::fma3(k, x[17], y[8]); y[17] = Ops::fma3(k, x[8], y[17]); }
      { k = Ops::fmac(w44, -0.2892857142857143, Ops::mulc(w35, 0.5785714285714286)); y[8] = Ops::fma3(k, x[18], y[8]); y[18] = Ops::fma3(k, x[8], y[18]); }
      { k = Ops::fmac(w29, -0.14464285714285716, Ops::mulc(w0, -0.2892857142857143)); y[8] = Ops::fma3(k, x[19], y[8]); y[19] = Ops::fma3(k, x[8], y[19]); }
      { k = Ops::fmac(w3, 1.1571428571428573, Ops::mulc(Lam[9], 1.4464285714285714)); y[9] = Ops::fma3(k, x[9], y[9]); }
      { k = Ops::mulc(w28, -0.14464285714285716); y[9] = Ops::fma3(k, x[10], y[9]); y[10] = Ops::fma3(k, x[9], y[10]); }
      { k = Ops::mulc(w28, -0.14464285714285716); y[9] = Ops::fma3(k, x[11], y[9]); y[11] = Ops::fma3(k, x[9], y[11]); }
      { k = Ops::fmac(w23, -0.14464285714285716, Ops::fmac(Lam[6], -0.2892857142857143, Ops::mulc(Lam[1], -0.43392857142857144))); y[9] = Ops::fma3(k, x[12], y[9]); y[12] = Ops::fma3(k, x[9], y[12]); }
      { k = Ops::fmac(w1, 0.5785714285714286, Ops::fmac(Lam[9], 0.7232142857142857, Ops::mulc(Lam[1], 1.1571428571428573))); y[9] = Ops::fma3(k, x[13], y[9]); y[13] = Ops::fma3(k, x[9], y[13]); }
      { k = Ops::fmac(w23, -0.14464285714285716, Ops::fmac(Lam[8], -0.2892857142857143, Ops::mulc(Lam[2], -0.43392857142857144))); y[9] = Ops::fma3(k, x[14], y[9]); y[14] = Ops::fma3(k, x[9], y[14]); }
      { k = Ops::fmac(w15, 0.5785714285714286, Ops::fmac(Lam[9], 0.7232142857142857, Ops::mulc(Lam[2], 1.1571428571428573))); y[9] = Ops::fma3(k, x[15], y[9]); y[15] = Ops::fma3(k, x[9], y[15]); }
      { k = Ops::fmac(w27, -0.14464285714285716, Ops::mulc(w10, -0.2892857142857143)); y[9] = Ops::fma3(k, x[16], y[9]); y[16] = Ops::fma3(k, x[9], y[16]); }
      { k = Ops::fmac(w54, 1.4464285714285714, Ops::mulc(w33, 0.5785714285714286)); y[9] = Ops::fma3(k, x[17], y[9]); y[17] = Ops::fma3(k, x[9], y[17]); }
      { k = Ops::fmac(w57, 1.4464285714285714, Ops::mulc(w34, 0.5785714285714286)); y[9] = Ops::fma3(k, x[18], y[9]); y[18] = Ops::fma3(k, x[9], y[18]); }
      { k = Ops::fmac(w23, -0.14464285714285716, Ops::fmac(w10, 0.7232142857142857, Ops::mulc(w0, 0.5785714285714286))); y[9] = Ops::fma3(k, x[19], y[9]); y[19] = Ops::fma3(k, x[9], y[19]); }
      { k = Ops::fmac(w24, 1.1571428571428573, Ops::mulc(Lam[4], 1.4464285714285714)); y[10] = Ops::fma3(k, x[10], y[10]); }
      { k = Ops::fmac(Lam[7], -0.43392857142857144, Ops::fmac(Lam[5], 0.2892857142857143, Ops::mulc(Lam[4], -0.43392857142857144))); y[10] = Ops::fma3(k, x[11], y[10]); y[11] = Ops::fma3(k, x[10], y[11]); }
      { k = Ops::fmac(w7, 0.5785714285714286, Ops::fmac(Lam[8], 1.1571428571428573, Ops::mulc(Lam[4], 0.7232142857142857))); y[10] = Ops::fma3(k, x[12], y[10]); y[12] = Ops::fma3(k, x[10], y[12]); }
      { k = Ops::fmac(w17, -0.14464285714285716, Ops::fmac(Lam[8], -0.43392857142857144, Ops::mulc(Lam[6], -0.2892857142857143))); y[10] = Ops::fma3(k, x[13], y[10]); y[13] = Ops::fma3(k, x[10], y[13]); }
      { k = Ops::fmac(w26, -0.14464285714285716, Ops::fmac(Lam[6], -0.43392857142857144, Ops::mulc(Lam[5], -0.2892857142857143))); y[10] = Ops::fma3(k, x[14], y[10]); y[14] = Ops::fma3(k, x[10], y[14]); }
      { k = Ops::mulc(w55, -0.2892857142857143); y[10] = Ops::fma3(k, x[15], y[10]); y[15] = Ops::fma3(k, x[10], y[15]); }
      { k = Ops::fmac(w46, 1.4464285714285714, Ops::mulc(w38, 0.5785714285714286)); y[10] = Ops::fma3(k, x[16], y[10]); y[16] = Ops::fma3(k, x[10], y[16]); }
      { k = Ops::fmac(w17, -0.14464285714285716, Ops::fmac(w14, 0.5785714285714286, Ops::mulc(w12, 0.7232142857142857))); y[10] = Ops::fma3(k, x[17], y[10]); y[17] = Ops::fma3(k, x[10], y[17]); }
      { k = Ops::fmac(w31, -0.14464285714285716, Ops::mulc(w12, -0.2892857142857143)); y[10] = Ops::fma3(k, x[18], y[10]); y[18] = Ops::fma3(k, x[10], y[18]); }
      { k = Ops::fmac(w51, -0.2892857142857143, Ops::mulc(w19, 0.5785714285714286)); y[10] = Ops::fma3(k, x[19], y[10]); y[19] = Ops::fma3(k, x[10], y[19]); }
      { k = Ops::fmac(w17, 1.1571428571428573, Ops::mulc(Lam[7], 1.4464285714285714)); y[11] = Ops::fma3(k, x[11], y[11]); }
      { k = Ops::fmac(w18, -0.14464285714285716, Ops::fmac(Lam[8], -0.43392857142857144, Ops::mulc(Lam[5], -0.2892857142857143))); y[11] = Ops::fma3(k, x[12], y[11]); y[12] = Ops::fma3(k, x[11], y[12]); }
      { k = Ops::fmac(w36, -0.14464285714285716, Ops::mulc(Lam[8], -0.2892857142857143)); y[11] = Ops::fma3(k, x[13], y[11]); y[13] = Ops::fma3(k, x[11], y[13]); }
      { k = Ops::fmac(w2, 0.5785714285714286, Ops::fmac(Lam[7], 0.7232142857142857, Ops::mulc(Lam[6], 1.1571428571428573))); y[11] = Ops::fma3(k, x[14], y[11]); y[14] = Ops::fma3(k, x[11], y[14]); }
      { k = Ops::fmac(w24, -0.14464285714285716, Ops::fmac(Lam[8], -0.2892857142857143, Ops::mulc(Lam[6], -0.43392857142857144))); y[11] = Ops::fma3(k, x[15], y[11]); y[15] = Ops::fma3(k, x[11], y[15]); }
      { k = Ops::fmac(w48, 1.4464285714285714, Ops::mulc(w37, 0.5785714285714286)); y[11] = Ops::fma3(k, x[16], y[11]); y[16] = Ops::fma3(k, x[11], y[16]); }
      { k = Ops::fmac(w42, -0.14464285714285716, Ops::mulc(w14, -0.2892857142857143)); y[11] = Ops::fma3(k, x[17], y[11]); y[17] = Ops::fma3(k, x[11], y[17]); }
      { k = Ops::fmac(w24, -0.14464285714285716, Ops::fmac(w14, 0.7232142857142857, Ops::mulc(w12, 0.5785714285714286))); y[11] = Ops::fma3(k, x[18], y[11]); y[18] = Ops::fma3(k, x[11], y[18]); }
      { k = Ops::fmac(w56, -0.2892857142857143, Ops::mulc(w36, 0.5785714285714286)); y[11] = Ops::fma3(k, x[19], y[11]); y[19] = Ops::fma3(k, x[11], y[19]); }
      { k = Ops::fmac(w25, 1.1571428571428573, Ops::mulc(Lam[4], 1.4464285714285714)); y[12] = Ops::fma3(k, x[12], y[12]); }
      { k = Ops::fmac(Lam[9], -0.43392857142857144, Ops::fmac(Lam[6], 0.2892857142857143, Ops::mulc(Lam[4], -0.43392857142857144))); y[12] = Ops::fma3(k, x[13], y[12]); y[13] = Ops::fma3(k, x[12], y[13]); }
      { k = Ops::fmac(w40, -0.14464285714285716, Ops::mulc(Lam[5], -0.2892857142857143)); y[12] = Ops::fma3(k, x[14], y[12]); y[14] = Ops::fma3(k, x[12], y[14]); }
      { k = Ops::fmac(w6, -0.14464285714285716, Ops::fmac(Lam[6], -0.2892857142857143, Ops::mulc(Lam[5], -0.43392857142857144))); y[12] = Ops::fma3(k, x[15], y[12]); y[15] = Ops::fma3(k, x[12], y[15]); }
      { k = Ops::fmac(w18, -0.14464285714285716, Ops::fmac(w15, 0.5785714285714286, Ops::mulc(w11, 0.7232142857142857))); y[12] = Ops::fma3(k, x[16], y[12]); y[16] = Ops::fma3(k, x[12], y[16]); }
      { k = Ops::fmac(w46, 1.4464285714285714, Ops::mulc(w20, 0.5785714285714286)); y[12] = Ops::fma3(k, x[17], y[12]); y[17] = Ops::fma3(k, x[12], y[17]); }
      { k = Ops::fmac(w29, -0.14464285714285716, Ops::mulc(w11, -0.2892857142857143)); y[12] = Ops::fma3(k, x[18], y[12]); y[18] = Ops::fma3(k, x[12], y[18]); }
      { k = Ops::fmac(w50, -0.2892857142857143, Ops::mulc(w40, 0.5785714285714286)); y[12] = Ops::fma3(k, x[19], y[12]); y[19] = Ops::fma3(k, x[12], y[19]); }
      { k = Ops::fmac(w18, 1.1571428571428573, Ops::mulc(Lam[9], 1.4464285714285714)); y[13] = Ops::fma3(k, x[13], y[13]); }
      { k = Ops::fmac(w25, -0.14464285714285716, Ops::fmac(Lam[8], -0.2892857142857143, Ops::mulc(Lam[5], -0.43392857142857144))); y[13] = Ops::fma3(k, x[14], y[13]); y[14] = Ops::fma3(k, x[13], y[14]); }
      { k = Ops::fmac(w10, 0.5785714285714286, Ops::fmac(Lam[9], 0.7232142857142857, Ops::mulc(Lam[5], 1.1571428571428573))); y[13] = Ops::fma3(k, x[15], y[13]); y[15] = Ops::fma3(k, x[13], y[15]); }
      { k = Ops::fmac(w42, -0.14464285714285716, Ops::mulc(w15, -0.2892857142857143)); y[13] = Ops::fma3(k, x[16], y[13]); y[16] = Ops::fma3(k, x[13], y[16]); }
      { k = Ops::fmac(w49, 1.4464285714285714, Ops::mulc(w39, 0.5785714285714286)); y[13] = Ops::fma3(k, x[17], y[13]); y[17] = Ops::fma3(k, x[13], y[17]); }
      { k = Ops::fmac(w25, -0.14464285714285716, Ops::fmac(w15, 0.7232142857142857, Ops::mulc(w11, 0.5785714285714286))); y[13] = Ops::fma3(k, x[18], y[13]); y[18] = Ops::fma3(k, x[13], y[18]); }
      { k = Ops::fmac(w57, 1.4464285714285714, Ops::mulc(w36, 0.5785714285714286)); y[13] = Ops::fma3(k, x[19], y[13]); y[19] = Ops::fma3(k, x[13], y[19]); }
      { k = Ops::fmac(w6, 1.1571428571428573, Ops::mulc(Lam[7], 1.4464285714285714)); y[14] = Ops::fma3(k, x[14], y[14]); }
      { k = Ops::fmac(Lam[9], -0.43392857142857144, Ops::fmac(Lam[8], 0.2892857142857143, Ops::mulc(Lam[7], -0.43392857142857144))); y[14] = Ops::fma3(k, x[15], y[14]); y[15] = Ops::fma3(k, x[14], y[15]); }
      { k = Ops::fmac(w26, -0.14464285714285716, Ops::fmac(w9, 0.7232142857142857, Ops::mulc(w1, 0.5785714285714286))); y[14] = Ops::fma3(k, x[16], y[14]); y[16] = Ops::fma3(k, x[14], y[16]); }
      { k = Ops::fmac(w29, -0.14464285714285716, Ops::mulc(w9, -0.2892857142857143)); y[14] = Ops::fma3(k, x[17], y[14]); y[17] = Ops::fma3(k, x[14], y[17]); }
      { k = Ops::fmac(w48, 1.4464285714285714, Ops::mulc(w35, 0.5785714285714286)); y[14] = Ops::fma3(k, x[18], y[14]); y[18] = Ops::fma3(k, x[14], y[18]); }
      { k = Ops::fmac(w52, 1.4464285714285714, Ops::mulc(w40, 0.5785714285714286)); y[14] = Ops::fma3(k, x[19], y[14]); y[19] = Ops::fma3(k, x[14], y[19]); }
      { k = Ops::fmac(w26, 1.1571428571428573, Ops::mulc(Lam[9], 1.4464285714285714)); y[15] = Ops::fma3(k, x[15], y[15]); }
      { k = Ops::fmac(w31, -0.14464285714285716, Ops::mulc(w1, -0.2892857142857143)); y[15] = Ops::fma3(k, x[16], y[15]); y[16] = Ops::fma3(k, x[15], y[16]); }
      { k = Ops::fmac(w9, 0.5785714285714286, Ops::fmac(w6, -0.14464285714285716, Ops::mulc(w1, 0.7232142857142857))); y[15] = Ops::fma3(k, x[17], y[15]); y[17] = Ops::fma3(k, x[15], y[17]); }
      { k = Ops::fmac(w49, 1.4464285714285714, Ops::mulc(w41, 0.5785714285714286)); y[15] = Ops::fma3(k, x[18], y[15]); y[18] = Ops::fma3(k, x[15], y[18]); }
      { k = Ops::fmac(w54, 1.4464285714285714, Ops::mulc(w19, 0.5785714285714286)); y[15] = Ops::fma3(k, x[19], y[15]); y[19] = Ops::fma3(k, x[15], y[19]); }
      { k = Ops::fmac(w59, 3.4714285714285715, Ops::mulc(Lam[7], 3.4714285714285715)); y[16] = Ops::fma3(k, x[16], y[16]); }
      { k = Ops::fmac(w59, 1.7357142857142858, Ops::fmac(w1, 1.7357142857142858, Ops::mulc(Lam[8], 3.4714285714285715))); y[16] = Ops::fma3(k, x[17], y[16]); y[17] = Ops::fma3(k, x[16], y[17]); }
      { k = Ops::fmac(w55, 3.4714285714285715, Ops::mulc(w27, 1.7357142857142858)); y[16] = Ops::fma3(k, x[18], y[16]); y[18] = Ops::fma3(k, x[16], y[18]); }
      { k = Ops::fmac(w60, 1.7357142857142858, Ops::fmac(w0, 1.7357142857142858, Ops::mulc(Lam[3], 3.4714285714285715))); y[16] = Ops::fma3(k, x[19], y[16]); y[19] = Ops::fma3(k, x[16], y[19]); }
      { k = Ops::fmac(w58, 3.4714285714285715, Ops::mulc(Lam[0], 3.4714285714285715)); y[17] = Ops::fma3(k, x[17], y[17]); }
      { k = Ops::fmac(w53, 3.4714285714285715, Ops::mulc(w29, 1.7357142857142858)); y[17] = Ops::fma3(k, x[18], y[17]); y[18] = Ops::fma3(k, x[17], y[18]); }
      { k = Ops::fmac(w58, 1.7357142857142858, Ops::fmac(w2, 1.7357142857142858, Ops::mulc(Lam[2], 3.4714285714285715))); y[17] = Ops::fma3(k, x[19], y[17]); y[19] = Ops::fma3(k, x[17], y[19]); }
      { k = Ops::fmac(w6, 3.4714285714285715, Ops::fmac(w5, 3.4714285714285715, Ops::mulc(w3, 3.4714285714285715))); y[18] = Ops::fma3(k, x[18], y[18]); }
      { k = Ops::fmac(w47, 3.4714285714285715, Ops::mulc(w31, 1.7357142857142858)); y[18] = Ops::fma3(k, x[19], y[18]); y[19] = Ops::fma3(k, x[18], y[19]); }
      { k = Ops::fmac(w60, 3.4714285714285715, Ops::mulc(Lam[9], 3.4714285714285715)); y[19] = Ops::fma3(k, x[19], y[19]); }
    }
    else if constexpr (MASS) {
      const typename Ops::T m0 = Ops::mulc(vol, 0.0035714285714285713);
      const typename Ops::T m1 = Ops::mulc(vol, 0.0004464285714285714);
      const typename Ops::T m2 = Ops::mulc(vol, -0.0026785714285714286);
      const typename Ops::T m3 = Ops::mulc(vol, 0.0013392857142857143);
      const typename Ops::T m4 = Ops::mulc(vol, 0.0006696428571428571);
      const typename Ops::T m5 = Ops::mulc(vol, 0.0040178571428571425);
      const typename Ops::T m6 = Ops::mulc(vol, 0.008035714285714285);
      const typename Ops::T m7 = Ops::mulc(vol, 0.024107142857142858);
      const typename Ops::T m8 = Ops::mulc(vol, -0.012053571428571429);
      const typename Ops::T m9 = Ops::mulc(vol, 0.012053571428571429);
      const typename Ops::T m10 = Ops::mulc(vol, -0.0060267857142857146);
      const typename Ops::T m11 = Ops::mulc(vol, 0.09642857142857143);
      const typename Ops::T m12 = Ops::mulc(vol, 0.048214285714285716);
      { k = m0; y[0] = Ops::mul(k, x[0]); }
      { k = m1; y[0] = Ops::fma3(k, x[1], y[0]); y[1] = Ops::mul(k, x[0]); }
      { k = m1; y[0] = Ops::fma3(k, x[2], y[0]); y[2] = Ops::mul(k, x[0]); }
      { k = m1; y[0] = Ops::fma3(k, x[3], y[0]); y[3] = Ops::mul(k, x[0]); }
      { k = m2; y[0] = Ops::fma3(k, x[4], y[0]); y[4] = Ops::mul(k, x[0]); }
      { k = m3; y[0] = Ops::fma3(k, x[5], y[0]); y[5] = Ops::mul(k, x[0]); }
      { k = m2; y[0] = Ops::fma3(k, x[6], y[0]); y[6] = Ops::mul(k, x[0]); }
      { k = m3; y[0] = Ops::fma3(k, x[7], y[0]); y[7] = Ops::mul(k, x[0]); }
      { k = m2; y[0] = Ops::fma3(k, x[8], y[0]); y[8] = Ops::mul(k, x[0]); }
      { k = m3; y[0] = Ops::fma3(k, x[9], y[0]); y[9] = Ops::mul(k, x[0]); }
      { k = m4; y[0] = Ops::fma3(k, x[10], y[0]); y[10] = Ops::mul(k, x[0]); }
      { k = m4; y[0] = Ops::fma3(k, x[11], y[0]); y[11] = Ops::mul(k, x[0]); }
      { k = m4; y[0] = Ops::fma3(k, x[12], y[0]); y[12] = Ops::mul(k, x[0]); }
      { k = m4; y[0] = Ops::fma3(k, x[13], y[0]); y[13] = Ops::mul(k, x[0]); }
      { k = m4; y[0] = Ops::fma3(k, x[14], y[0]); y[14] = Ops::mul(k, x[0]); }
      { k = m4; y[0] = Ops::fma3(k, x[15], y[0]); y[15] = Ops::mul(k, x[0]); }
      { k = m5; y[0] = Ops::fma3(k, x[16], y[0]); y[16] = Ops::mul(k, x[0]); }
      { k = m5; y[0] = Ops::fma3(k, x[17], y[0]); y[17] = Ops::mul(k, x[0]); }
      { k = m5; y[0] = Ops::fma3(k, x[18], y[0]); y[18] = Ops::mul(k, x[0]); }
      { k = m6; y[0] = Ops::fma3(k, x[19], y[0]); y[19] = Ops::mul(k, x[0]); }
      { k = m0; y[1] = Ops::fma3(k, x[1], y[1]); }
      { k = m1; y[1] = Ops::fma3(k, x[2], y[1]); y[2] = Ops::fma3(k, x[1], y[2]); }
      { k = m1; y[1] = Ops::fma3(k, x[3], y[1]); y[3] = Ops::fma3(k, x[1], y[3]); }
      { k = m3; y[1] = Ops::fma3(k, x[4], y[1]); y[4] = Ops::fma3(k, x[1], y[4]); }
      { k = m2; y[1] = Ops::fma3(k, x[5], y[1]); y[5] = Ops::fma3(k, x[1], y[5]); }
      { k = m4; y[1] = Ops::fma3(k, x[6], y[1]); y[6] = Ops::fma3(k, x[1], y[6]); }
      { k = m4; y[1] = Ops::fma3(k, x[7], y[1]); y[7] = Ops::fma3(k, x[1], y[7]); }
      { k = m4; y[1] = Ops::fma3(k, x[8], y[1]); y[8] = Ops::fma3(k, x[1], y[8]); }
      { k = m4; y[1] = Ops::fma3(k, x[9], y[1]); y[9] = Ops::fma3(k, x[1], y[9]); }
      { k = m2; y[1] = Ops::fma3(k, x[10], y[1]); y[10] = Ops::fma3(k, x[1], y[10]); }
      { k = m3; y[1] = Ops::fma3(k, x[11], y[1]); y[11] = Ops::fma3(k, x[1], y[11]); }
      { k = m2; y[1] = Ops::fma3(k, x[12], y[1]); y[12] = Ops::fma3(k, x[1], y[12]); }
      { k = m3; y[1] = Ops::fma3(k, x[13], y[1]); y[13] = Ops::fma3(k, x[1], y[13]); }
      { k = m4; y[1] = Ops::fma3(k, x[14], y[1]); y[14] = Ops::fma3(k, x[1], y[14]); }
      { k = m4; y[1] = Ops::fma3(k, x[15], y[1]); y[15] = Ops::fma3(k, x[1], y[15]); }
      { k = m5; y[1] = Ops::fma3(k, x[16], y[1]); y[16] = Ops::fma3(k, x[1], y[16]); }
      { k = m5; y[1] = Ops::fma3(k, x[17], y[1]); y[17] = Ops::fma3(k, x[1], y[17]); }
      { k = m6; y[1] = Ops::fma3(k, x[18], y[1]); y[18] = Ops::fma3(k, x[1], y[18]); }
      { k = m5; y[1] = Ops::fma3(k, x[19], y[1]); y[19] = Ops::fma3(k, x[1], y[19]); }
      { k = m0; y[2] = Ops::fma3(k, x[2], y[2]); }
      { k = m1; y[2] = Ops::fma3(k, x[3], y[2]); y[3] = Ops::fma3(k, x[2], y[3]); }
      { k = m4; y[2] = Ops::fma3(k, x[4], y[2]); y[4] = Ops::fma3(k, x[2], y[4]); }
      { k = m4; y[2] = Ops::fma3(k, x[5], y[2]); y[5] = Ops::fma3(k, x[2], y[5]); }
      { k = m3; y[2] = Ops::fma3(k, x[6], y[2]); y[6] = Ops::fma3(k, x[2], y[6]); }
      { k = m2; y[2] = Ops::fma3(k, x[7], y[2]); y[7] = Ops::fma3(k, x[2], y[7]); }
      { k = m4; y[2] = Ops::fma3(k, x[8], y[2]); y[8] = Ops::fma3(k, x[2], y[8]); }
      { k = m4; y[2] = Ops::fma3(k, x[9], y[2]); y[9] = Ops::fma3(k, x[2], y[9]); }
      { k = m3; y[2] = Ops::fma3(k, x[10], y[2]); y[10] = Ops::fma3(k, x[2], y[10]); }
      { k = m2; y[2] = Ops::fma3(k, x[11], y[2]); y[11] = Ops::fma3(k, x[2], y[11]); }
      { k = m4; y[2] = Ops::fma3(k, x[12], y[2]); y[12] = Ops::fma3(k, x[2], y[12]); }
      { k = m4; y[2] = Ops::fma3(k, x[13], y[2]); y[13] = Ops::fma3(k, x[2], y[13]); }
      { k = m2; y[2] = Ops::fma3(k, x[14], y[2]); y[14] = Ops::fma3(k, x[2], y[14]); }
      { k = m3; y[2] = Ops::fma3(k, x[15], y[2]); y[15] = Ops::fma3(k, x[2], y[15]); }
      { k = m5; y[2] = Ops::fma3(k, x[16], y[2]); y[16] = Ops::fma3(k, x[2], y[16]); }
      { k = m6; y[2] = Ops::fma3(k, x[17], y[2]); y[17] = Ops::fma3(k, x[2], y[17]); }
      { k = m5; y[2] = Ops::fma3(k, x[18], y[2]); y[18] = Ops::fma3(k, x[2], y[18]); }
      { k = m5; y[2] = Ops::fma3(k, x[19], y[2]); y[19] = Ops::fma3(k, x[2], y[19]); }
      { k = m0; y[3] = Ops::fma3(k, x[3], y[3]); }
      { k = m4; y[3] = Ops::fma3(k, x[4], y[3]); y[4] = Ops::fma3(k, x[3], y[4]); }
      { k = m4; y[3] = Ops::fma3(k, x[5], y[3]); y[5] = Ops::fma3(k, x[3], y[5]); }
      { k = m4; y[3] = Ops::fma3(k, x[6], y[3]); y[6] = Ops::fma3(k, x[3], y[6]); }
      { k = m4; y[3] = Ops::fma3(k, x[7], y[3]); y[7] = Ops::fma3(k, x[3], y[7]); }
      { k = m3; y[3] = Ops::fma3(k, x[8], y[3]); y[8] = Ops::fma3(k, x[3], y[8]); }
      { k = m2; y[3] = Ops::fma3(k, x[9], y[3]); y[9] = Ops::fma3(k, x[3], y[9]); }
      { k = m4; y[3] = Ops::fma3(k, x[10], y[3]); y[10] = Ops::fma3(k, x[3], y[10]); }
      { k = m4; y[3] = Ops::fma3(k, x[11], y[3]); y[11] = Ops::fma3(k, x[3], y[11]); }
      { k = m3; y[3] = Ops::fma3(k, x[12], y[3]); y[12] = Ops::fma3(k, x[3], y[12]); }
      { k = m2; y[3] = Ops::fma3(k, x[13], y[3]); y[13] = Ops::fma3(k, x[3], y[13]); }
      { k = m3; y[3] = Ops::fma3(k, x[14], y[3]); y[14] = Ops::fma3(k, x[3], y[14]); }
      { k = m2; y[3] = Ops::fma3(k, x[15], y[3]); y[15] = Ops::fma3(k, x[3], y[15]); }
      { k = m6; y[3] = Ops::fma3(k, x[16], y[3]); y[16] = Ops::fma3(k, x[3], y[16]); }
      { k = m5; y[3] = Ops::fma3(k, x[17], y[3]); y[17] = Ops::fma3(k, x[3], y[17]); }
      { k = m5; y[3] = Ops::fma3(k, x[18], y[3]); y[18] = Ops::fma3(k, x[3], y[18]); }
      { k = m5; y[3] = Ops::fma3(k, x[19], y[3]); y[19] = Ops::fma3(k, x[3], y[19]); }
      { k = m7; y[4] = Ops::fma3(k, x[4], y[4]); }
      { k = m8; y[4] = Ops::fma3(k, x[5], y[4]); y[5] = Ops::fma3(k, x[4], y[5]); }
      { k = m9; y[4] = Ops::fma3(k, x[6], y[4]); y[6] = Ops::fma3(k, x[4], y[6]); }
      { k = m10; y[4] = Ops::fma3(k, x[7], y[4]); y[7] = Ops::fma3(k, x[4], y[7]); }
      { k = m9; y[4] = Ops::fma3(k, x[8], y[4]); y[8] = Ops::fma3(k, x[4], y[8]); }
      { k = m10; y[4] = Ops::fma3(k, x[9], y[4]); y[9] = Ops::fma3(k, x[4], y[9]); }
      { k = m10; y[4] = Ops::fma3(k, x[10], y[4]); y[10] = Ops::fma3(k, x[4], y[10]); }
      { k = m10; y[4] = Ops::fma3(k, x[12], y[4]); y[12] = Ops::fma3(k, x[4], y[12]); }
      { k = m8; y[4] = Ops::fma3(k, x[19], y[4]); y[19] = Ops::fma3(k, x[4], y[19]); }
      { k = m7; y[5] = Ops::fma3(k, x[5], y[5]); }
      { k = m10; y[5] = Ops::fma3(k, x[6], y[5]); y[6] = Ops::fma3(k, x[5], y[6]); }
      { k = m10; y[5] = Ops::fma3(k, x[8], y[5]); y[8] = Ops::fma3(k, x[5], y[8]); }
      { k = m9; y[5] = Ops::fma3(k, x[10], y[5]); y[10] = Ops::fma3(k, x[5], y[10]); }
      { k = m10; y[5] = Ops::fma3(k, x[11], y[5]); y[11] = Ops::fma3(k, x[5], y[11]); }
      { k = m9; y[5] = Ops::fma3(k, x[12], y[5]); y[12] = Ops::fma3(k, x[5], y[12]); }
      { k = m10; y[5] = Ops::fma3(k, x[13], y[5]); y[13] = Ops::fma3(k, x[5], y[13]); }
      { k = m8; y[5] = Ops::fma3(k, x[18], y[5]); y[18] = Ops::fma3(k, x[5], y[18]); }
      { k = m7; y[6] = Ops::fma3(k, x[6], y[6]); }
      { k = m8; y[6] = Ops::fma3(k, x[7], y[6]); y[7] = Ops::fma3(k, x[6], y[7]); }
      { k = m9; y[6] = Ops::fma3(k, x[8], y[6]); y[8] = Ops::fma3(k, x[6], y[8]); }
      { k = m10; y[6] = Ops::fma3(k, x[9], y[6]); y[9] = Ops::fma3(k, x[6], y[9]); }
      { k = m10; y[6] = Ops::fma3(k, x[11], y[6]); y[11] = Ops::fma3(k, x[6], y[11]); }
      { k = m10; y[6] = Ops::fma3(k, x[14], y[6]); y[14] = Ops::fma3(k, x[6], y[14]); }
      { k = m8; y[6] = Ops::fma3(k, x[19], y[6]); y[19] = Ops::fma3(k, x[6], y[19]); }
      { k = m7; y[7] = Ops::fma3(k, x[7], y[7]); }
      { k = m10; y[7] = Ops::fma3(k, x[8], y[7]); y[8] = Ops::fma3(k, x[7], y[8]); }
      { k = m10; y[7] = Ops::fma3(k, x[10], y[7]); y[10] = Ops::fma3(k, x[7], y[10]); }
      { k = m9; y[7] = Ops::fma3(k, x[11], y[7]); y[11] = Ops::fma3(k, x[7], y[11]); }
      { k = m9; y[7] = Ops::fma3(k, x[14], y[7]); y[14] = Ops::fma3(k, x[7], y[14]); }
      { k = m10; y[7] = Ops::fma3(k, x[15], y[7]); y[15] = Ops::fma3(k, x[7], y[15]); }
      { k = m8; y[7] = Ops::fma3(k, x[17], y[7]); y[17] = Ops::fma3(k, x[7], y[17]); }
      { k = m7; y[8] = Ops::fma3(k, x[8], y[8]); }
      { k = m8; y[8] = Ops::fma3(k, x[9], y[8]); y[9] = Ops::fma3(k, x[8], y[9]); }
      { k = m10; y[8] = Ops::fma3(k, x[13], y[8]); y[13] = Ops::fma3(k, x[8], y[13]); }
      { k = m10; y[8] = Ops::fma3(k, x[15], y[8]); y[15] = Ops::fma3(k, x[8], y[15]); }
      { k = m8; y[8] = Ops::fma3(k, x[19], y[8]); y[19] = Ops::fma3(k, x[8], y[19]); }
      { k = m7; y[9] = Ops::fma3(k, x[9], y[9]); }
      { k = m10; y[9] = Ops::fma3(k, x[12], y[9]); y[12] = Ops::fma3(k, x[9], y[12]); }
      { k = m9; y[9] = Ops::fma3(k, x[13], y[9]); y[13] = Ops::fma3(k, x[9], y[13]); }
      { k = m10; y[9] = Ops::fma3(k, x[14], y[9]); y[14] = Ops::fma3(k, x[9], y[14]); }
      { k = m9; y[9] = Ops::fma3(k, x[15], y[9]); y[15] = Ops::fma3(k, x[9], y[15]); }
      { k = m8; y[9] = Ops::fma3(k, x[16], y[9]); y[16] = Ops::fma3(k, x[9], y[16]); }
      { k = m7; y[10] = Ops::fma3(k, x[10], y[10]); }
      { k = m8; y[10] = Ops::fma3(k, x[11], y[10]); y[11] = Ops::fma3(k, x[10], y[11]); }
      { k = m9; y[10] = Ops::fma3(k, x[12], y[10]); y[12] = Ops::fma3(k, x[10], y[12]); }
      { k = m10; y[10] = Ops::fma3(k, x[13], y[10]); y[13] = Ops::fma3(k, x[10], y[13]); }
      { k = m10; y[10] = Ops::fma3(k, x[14], y[10]); y[14] = Ops::fma3(k, x[10], y[14]); }
      { k = m8; y[10] = Ops::fma3(k, x[18], y[10]); y[18] = Ops::fma3(k, x[10], y[18]); }
      { k = m7; y[11] = Ops::fma3(k, x[11], y[11]); }
      { k = m10; y[11] = Ops::fma3(k, x[12], y[11]); y[12] = Ops::fma3(k, x[11], y[12]); }
      { k = m9; y[11] = Ops::fma3(k, x[14], y[11]); y[14] = Ops::fma3(k, x[11], y[14]); }
      { k = m10; y[11] = Ops::fma3(k, x[15], y[11]); y[15] = Ops::fma3(k, x[11], y[15]); }
      { k = m8; y[11] = Ops::fma3(k, x[17], y[11]); y[17] = Ops::fma3(k, x[11], y[17]); }
      { k = m7; y[12] = Ops::fma3(k, x[12], y[12]); }
      { k = m8; y[12] = Ops::fma3(k, x[13], y[12]); y[13] = Ops::fma3(k, x[12], y[13]); }
      { k = m10; y[12] = Ops::fma3(k, x[15], y[12]); y[15] = Ops::fma3(k, x[12], y[15]); }
      { k = m8; y[12] = Ops::fma3(k, x[18], y[12]); y[18] = Ops::fma3(k, x[12], y[18]); }
      { k = m7; y[13] = Ops::fma3(k, x[13], y[13]); }
      { k = m10; y[13] = Ops::fma3(k, x[14], y[13]); y[14] = Ops::fma3(k, x[13], y[14]); }
      { k = m9; y[13] = Ops::fma3(k, x[15], y[13]); y[15] = Ops::fma3(k, x[13], y[15]); }
      { k = m8; y[13] = Ops::fma3(k, x[16], y[13]); y[16] = Ops::fma3(k, x[13], y[16]); }
      { k = m7; y[14] = Ops::fma3(k, x[14], y[14]); }
      { k = m8; y[14] = Ops::fma3(k, x[15], y[14]); y[15] = Ops::fma3(k, x[14], y[15]); }
      { k = m8; y[14] = Ops::fma3(k, x[17], y[14]); y[17] = Ops::fma3(k, x[14], y[17]); }
      { k = m7; y[15] = Ops::fma3(k, x[15], y[15]); }
      { k = m8; y[15] = Ops::fma3(k, x[16], y[15]); y[16] = Ops::fma3(k, x[15], y[16]); }
      { k = m11; y[16] = Ops::fma3(k, x[16], y[16]); }
      { k = m12; y[16] = Ops::fma3(k, x[17], y[16]); y[17] = Ops::fma3(k, x[16], y[17]); }
      { k = m12; y[16] = Ops::fma3(k, x[18], y[16]); y[18] = Ops::fma3(k, x[16], y[18]); }
      { k = m12; y[16] = Ops::fma3(k, x[19], y[16]); y[19] = Ops::fma3(k, x[16], y[19]); }
      { k = m11; y[17] = Ops::fma3(k, x[17], y[17]); }
      { k = m12; y[17] = Ops::fma3(k, x[18], y[17]); y[18] = Ops::fma3(k, x[17], y[18]); }
      { k = m12; y[17] = Ops::fma3(k, x[19], y[17]); y[19] = Ops::fma3(k, x[17], y[19]); }
      { k = m11; y[18] = Ops::fma3(k, x[18], y[18]); }
      { k = m12; y[18] = Ops::fma3(k, x[19], y[18]); y[19] = Ops::fma3(k, x[18], y[19]); }
      { k = m11; y[19] = Ops::fma3(k, x[19], y[19]); }
    }
  }
  __host__ __device__ static constexpr int upper_index(int i, int j) {
    return i <= j ? i * 20 - (i * (i - 1)) / 2 + (j - i) : j * 20 - (j * (j - 1)) / 2 + (i - j);
  }
};

template <> struct Source<2, 1, 1> {
  static constexpr int ND = 3;
  static constexpr int NF = 3;
  // b_i = vol * sum_k Mx[i][k] f_k
  template <class Ops> __device__ __forceinline__ static void vec(const typename Ops::T& vol, const typename Ops::T* f, typename Ops::T* b) {
    b[0] = Ops::mul(vol, Ops::fmac(f[2], 0.08333333333333333, Ops::fmac(f[1], 0.08333333333333333, Ops::mulc(f[0], 0.16666666666666666))));
    b[1] = Ops::mul(vol, Ops::fmac(f[2], 0.08333333333333333, Ops::fmac(f[1], 0.16666666666666666, Ops::mulc(f[0], 0.08333333333333333))));
    b[2] = Ops::mul(vol, Ops::fmac(f[2], 0.16666666666666666, Ops::fmac(f[1], 0.08333333333333333, Ops::mulc(f[0], 0.08333333333333333))));
  }
};

template <> struct Source<2, 2, 2> {
  static constexpr int ND = 6;
  static constexpr int NF = 6;
  // b_i = vol * sum_k Mx[i][k] f_k
  template <class Ops> __device__ __forceinline__ static void vec(const typename Ops::T& vol, const typename Ops::T* f, typename Ops::T* b) {
    b[0] = Ops::mul(vol, Ops::fmac(f[5], -0.022222222222222223, Ops::fmac(f[2], -0.005555555555555556, Ops::fmac(f[1], -0.005555555555555556, Ops::mulc(f[0], 0.03333333333333333)))));
    b[1] = Ops::mul(vol, Ops::fmac(f[4], -0.022222222222222223, Ops::fmac(f[2], -0.005555555555555556, Ops::fmac(f[1], 0.03333333333333333, Ops::mulc(f[0], -0.005555555555555556)))));
    b[2] = Ops::mul(vol, Ops::fmac(f[3], -0.022222222222222223, Ops::fmac(f[2], 0.03333333333333333, Ops::fmac(f[1], -0.005555555555555556, Ops::mulc(f[0], -0.005555555555555556)))));
    b[3] = Ops::mul(vol, Ops::fmac(f[5], 0.08888888888888889, Ops::fmac(f[4], 0.08888888888888889, Ops::fmac(f[3], 0.17777777777777778, Ops::mulc(f[2], -0.022222222222222223)))));
    b[4] = Ops::mul(vol, Ops::fmac(f[5], 0.08888888888888889, Ops::fmac(f[4], 0.17777777777777778, Ops::fmac(f[3], 0.08888888888888889, Ops::mulc(f[1], -0.022222222222222223)))));
    b[5] = Ops::mul(vol, Ops::fmac(f[5], 0.17777777777777778, Ops::fmac(f[4], 0.08888888888888889, Ops::fmac(f[3], 0.08888888888888889, Ops::mulc(f[0], -0.022222222222222223)))));
  }
};

template <> struct Source<2, 2, 1> {
  static constexpr int ND = 6;
  static constexpr int NF = 3;
  // b_i = vol * sum_k Mx[i][k] f_k
  template <class Ops> __device__ __forceinline__ static void vec(const typename Ops::T& vol, const typename Ops::T* f, typename Ops::T* b) {
    b[0] = Ops::mul(vol, Ops::fmac(f[2], -0.016666666666666666, Ops::fmac(f[1], -0.016666666666666666, Ops::mulc(f[0], 0.03333333333333333))));
    b[1] = Ops::mul(vol, Ops::fmac(f[2], -0.016666666666666666, Ops::fmac(f[1], 0.03333333333333333, Ops::mulc(f[0], -0.016666666666666666))));
    b[2] = Ops::mul(vol, Ops::fmac(f[2], 0.03333333333333333, Ops::fmac(f[1], -0.016666666666666666, Ops::mulc(f[0], -0.016666666666666666))));
    b[3] = Ops::mul(vol, Ops::fmac(f[2], 0.06666666666666667, Ops::fmac(f[1], 0.13333333333333333, Ops::mulc(f[0], 0.13333333333333333))));
    b[4] = Ops::mul(vol, Ops::fmac(f[2], 0.13333333333333333, Ops::fmac(f[1], 0.06666666666666667, Ops::mulc(f[0], 0.13333333333333333))));
    b[5] = Ops::mul(vol, Ops::fmac(f[2], 0.13333333333333333, Ops::fmac(f[1], 0.13333333333333333, Ops::mulc(f[0], 0.06666666666666667))));
  }
};

template <> struct Source<2, 4, 1> {
  static constexpr int ND = 15;
  static constexpr int NF = 3;
  // b_i = vol * sum_k Mx[i][k] f_k
  template <class Ops> __device__ __forceinline__ static void vec(const typename Ops::T& vol, const typename Ops::T* f, typename Ops::T* b) {
    b[0] = Ops::mul(vol, Ops::fmac(f[2], -0.003968253968253968, Ops::fmac(f[1], -0.003968253968253968, Ops::mulc(f[0], 0.007936507936507936))));
    b[1] = Ops::mul(vol, Ops::fmac(f[2], -0.003968253968253968, Ops::fmac(f[1], 0.007936507936507936, Ops::mulc(f[0], -0.003968253968253968))));
    b[2] = Ops::mul(vol, Ops::fmac(f[2], 0.007936507936507936, Ops::fmac(f[1], -0.003968253968253968, Ops::mulc(f[0], -0.003968253968253968))));
    b[3] = Ops::mul(vol, Ops::fmac(f[2], 0.012698412698412698, Ops::fmac(f[1], 0.025396825396825397, Ops::mulc(f[0], 0.050793650793650794))));
    b[4] = Ops::mul(vol, Ops::fmac(f[2], -0.009523809523809525, Ops::fmac(f[1], -0.006349206349206349, Ops::mulc(f[0], -0.006349206349206349))));
    b[5] = Ops::mul(vol, Ops::fmac(f[2], 0.012698412698412698, Ops::fmac(f[1], 0.050793650793650794, Ops::mulc(f[0], 0.025396825396825397))));
    b[6] = Ops::mul(vol, Ops::fmac(f[2], 0.025396825396825397, Ops::fmac(f[1], 0.012698412698412698, Ops::mulc(f[0], 0.050793650793650794))));
    b[7] = Ops::mul(vol, Ops::fmac(f[2], -0.006349206349206349, Ops::fmac(f[1], -0.009523809523809525, Ops::mulc(f[0], -0.006349206349206349))));
    b[8] = Ops::mul(vol, Ops::fmac(f[2], 0.050793650793650794, Ops::fmac(f[1], 0.012698412698412698, Ops::mulc(f[0], 0.025396825396825397))));
    b[9] = Ops::mul(vol, Ops::fmac(f[2], 0.025396825396825397, Ops::fmac(f[1], 0.050793650793650794, Ops::mulc(f[0], 0.012698412698412698))));
    b[10] = Ops::mul(vol, Ops::fmac(f[2], -0.006349206349206349, Ops::fmac(f[1], -0.006349206349206349, Ops::mulc(f[0], -0.009523809523809525))));
    b[11] = Ops::mul(vol, Ops::fmac(f[2], 0.050793650793650794, Ops::fmac(f[1], 0.025396825396825397, Ops::mulc(f[0], 0.012698412698412698))));
    b[12] = Ops::mul(vol, Ops::fmac(f[2], 0.025396825396825397, Ops::fmac(f[1], 0.025396825396825397, Ops::mulc(f[0], 0.12698412698412698))));
    b[13] = Ops::mul(vol, Ops::fmac(f[2], 0.025396825396825397, Ops::fmac(f[1], 0.12698412698412698, Ops::mulc(f[0], 0.025396825396825397))));
    b[14] = Ops::mul(vol, Ops::fmac(f[2], 0.12698412698412698, Ops::fmac(f[1], 0.025396825396825397, Ops::mulc(f[0], 0.025396825396825397))));
  }
};

template <> struct Source<3, 1, 1> {
  static constexpr int ND = 4;
  static constexpr int NF = 4;
  // b_i = vol * sum_k Mx[i][k] f_k
  template <class Ops> __device__ __forceinline__ static void vec(const typename Ops::T& vol, const typename Ops::T* f, typename Ops::T* b) {
    b[0] = Ops::mul(vol, Ops::fmac(f[3], 0.05, Ops::fmac(f[2], 0.05, Ops::fmac(f[1], 0.05, Ops::mulc(f[0], 0.1)))));
    b[1] = Ops::mul(vol, Ops::fmac(f[3], 0.05, Ops::fmac(f[2], 0.05, Ops::fmac(f[1], 0.1, Ops::mulc(f[0], 0.05)))));
    b[2] = Ops::mul(vol, Ops::fmac(f[3], 0.05, Ops::fmac(f[2], 0.1, Ops::fmac(f[1], 0.05, Ops::mulc(f[0], 0.05)))));
    b[3] = Ops::mul(vol, Ops::fmac(f[3], 0.1, Ops::fmac(f[2], 0.05, Ops::fmac(f[1], 0.05, Ops::mulc(f[0], 0.05)))));
  }
};

template <> struct Source<3, 2, 2> {
  static constexpr int ND = 10;
  static constexpr int NF = 10;
  // b_i = vol * sum_k Mx[i][k] f_k
  template <class Ops> __device__ __forceinline__ static void vec(const typename Ops::T& vol, const typename Ops::T* f, typename Ops::T* b) {
    b[0] = Ops::mul(vol, Ops::fmac(f[9], -0.014285714285714285, Ops::fmac(f[8], -0.014285714285714285, Ops::fmac(f[7], -0.014285714285714285, Ops::fmac(f[6], -0.009523809523809525, Ops::fmac(f[5], -0.009523809523809525, Ops::fmac(f[4], -0.009523809523809525, Ops::fmac(f[3], 0.002380952380952381, Ops::fmac(f[2], 0.002380952380952381, Ops::fmac(f[1], 0.002380952380952381, Ops::mulc(f[0], 0.014285714285714285)))))))))));
    b[1] = Ops::mul(vol, Ops::fmac(f[9], -0.014285714285714285, Ops::fmac(f[8], -0.009523809523809525, Ops::fmac(f[7], -0.009523809523809525, Ops::fmac(f[6], -0.014285714285714285, Ops::fmac(f[5], -0.014285714285714285, Ops::fmac(f[4], -0.009523809523809525, Ops::fmac(f[3], 0.002380952380952381, Ops::fmac(f[2], 0.002380952380952381, Ops::fmac(f[1], 0.014285714285714285, Ops::mulc(f[0], 0.002380952380952381)))))))))));
    b[2] = Ops::mul(vol, Ops::fmac(f[9], -0.009523809523809525, Ops::fmac(f[8], -0.014285714285714285, Ops::fmac(f[7], -0.009523809523809525, Ops::fmac(f[6], -0.014285714285714285, Ops::fmac(f[5], -0.009523809523809525, Ops::fmac(f[4], -0.014285714285714285, Ops::fmac(f[3], 0.002380952380952381, Ops::fmac(f[2], 0.014285714285714285, Ops::fmac(f[1], 0.002380952380952381, Ops::mulc(f[0], 0.002380952380952381)))))))))));
    b[3] = Ops::mul(vol, Ops::fmac(f[9], -0.009523809523809525, Ops::fmac(f[8], -0.009523809523809525, Ops::fmac(f[7], -0.014285714285714285, Ops::fmac(f[6], -0.009523809523809525, Ops::fmac(f[5], -0.014285714285714285, Ops::fmac(f[4], -0.014285714285714285, Ops::fmac(f[3], 0.014285714285714285, Ops::fmac(f[2], 0.002380952380952381, Ops::fmac(f[1], 0.002380952380952381, Ops::mulc(f[0], 0.002380952380952381)))))))))));
    b[4] = Ops::mul(vol, Ops::fmac(f[9], 0.01904761904761905, Ops::fmac(f[8], 0.0380952380952381, Ops::fmac(f[7], 0.0380952380952381, Ops::fmac(f[6], 0.0380952380952381, Ops::fmac(f[5], 0.0380952380952381, Ops::fmac(f[4], 0.0761904761904762, Ops::fmac(f[3], -0.014285714285714285, Ops::fmac(f[2], -0.014285714285714285, Ops::fmac(f[1], -0.009523809523809525, Ops::mulc(f[0], -0.009523809523809525)))))))))));
    b[5] = Ops::mul(vol, Ops::fmac(f[9], 0.0380952380952381, Ops::fmac(f[8], 0.01904761904761905, Ops::fmac(f[7], 0.0380952380952381, Ops::fmac(f[6], 0.0380952380952381, Ops::fmac(f[5], 0.0761904761904762, Ops::fmac(f[4], 0.0380952380952381, Ops::fmac(f[3], -0.014285714285714285, Ops::fmac(f[2], -0.009523809523809525, Ops::fmac(f[1], -0.014285714285714285, Ops::mulc(f[0], -0.009523809523809525)))))))))));
    b[6] = Ops::mul(vol, Ops::fmac(f[9], 0.0380952380952381, Ops::fmac(f[8], 0.0380952380952381, Ops::fmac(f[7], 0.01904761904761905, Ops::fmac(f[6], 0.0761904761904762, Ops::fmac(f[5], 0.0380952380952381, Ops::fmac(f[4], 0.0380952380952381, Ops::fmac(f[3], -0.009523809523809525, Ops::fmac(f[2], -0.014285714285714285, Ops::fmac(f[1], -0.014285714285714285, Ops::mulc(f[0], -0.009523809523809525)))))))))));
    b[7] = Ops::mul(vol, Ops::fmac(f[9], 0.0380952380952381, Ops::fmac(f[8], 0.0380952380952381, Ops::fmac(f[7], 0.0761904761904762, Ops::fmac(f[6], 0.01904761904761905, Ops::fmac(f[5], 0.0380952380952381, Ops::fmac(f[4], 0.0380952380952381, Ops::fmac(f[3], -0.014285714285714285, Ops::fmac(f[2], -0.009523809523809525, Ops::fmac(f[1], -0.009523809523809525, Ops::mulc(f[0], -0.014285714285714285)))))))))));
    b[8] = Ops::mul(vol, Ops::fmac(f[9], 0.0380952380952381, Ops::fmac(f[8], 0.0761904761904762, Ops::fmac(f[7], 0.0380952380952381, Ops::fmac(f[6], 0.0380952380952381, Ops::fmac(f[5], 0.01904761904761905, Ops::fmac(f[4], 0.0380952380952381, Ops::fmac(f[3], -0.009523809523809525, Ops::fmac(f[2], -0.014285714285714285, Ops::fmac(f[1], -0.009523809523809525, Ops::mulc(f[0], -0.014285714285714285)))))))))));
    b[9] = Ops::mul(vol, Ops::fmac(f[9], 0.0761904761904762, Ops::fmac(f[8], 0.0380952380952381, Ops::fmac(f[7], 0.0380952380952381, Ops::fmac(f[6], 0.0380952380952381, Ops::fmac(f[5], 0.0380952380952381, Ops::fmac(f[4], 0.01904761904761905, Ops::fmac(f[3], -0.009523809523809525, Ops::fmac(f[2], -0.009523809523809525, Ops::fmac(f[1], -0.014285714285714285, Ops::mulc(f[0], -0.014285714285714285)))))))))));
  }
};

template <> struct Source<3, 2, 1> {
  static constexpr int ND = 10;
  static constexpr int NF = 4;
  // b_i = vol * sum_k Mx[i][k] f_k
  template <class Ops> __device__ __forceinline__ static void vec(const typename Ops::T& vol, const typename Ops::T* f, typename Ops::T* b) {
    b[0] = Ops::mul(vol, Ops::fmac(f[3], -0.016666666666666666, Ops::fmac(f[2], -0.016666666666666666, Ops::mulc(f[1], -0.016666666666666666))));
    b[1] = Ops::mul(vol, Ops::fmac(f[3], -0.016666666666666666, Ops::fmac(f[2], -0.016666666666666666, Ops::mulc(f[0], -0.016666666666666666))));
    b[2] = Ops::mul(vol, Ops::fmac(f[3], -0.016666666666666666, Ops::fmac(f[1], -0.016666666666666666, Ops::mulc(f[0], -0.016666666666666666))));
    b[3] = Ops::mul(vol, Ops::fmac(f[2], -0.016666666666666666, Ops::fmac(f[1], -0.016666666666666666, Ops::mulc(f[0], -0.016666666666666666))));
    b[4] = Ops::mul(vol, Ops::fmac(f[3], 0.03333333333333333, Ops::fmac(f[2], 0.03333333333333333, Ops::fmac(f[1], 0.06666666666666667, Ops::mulc(f[0], 0.06666666666666667)))));
    b[5] = Ops::mul(vol, Ops::fmac(f[3], 0.03333333333333333, Ops::fmac(f[2], 0.06666666666666667, Ops::fmac(f[1], 0.03333333333333333, Ops::mulc(f[0], 0.06666666666666667)))));
    b[6] = Ops::mul(vol, Ops::fmac(f[3], 0.06666666666666667, Ops::fmac(f[2], 0.03333333333333333, Ops::fmac(f[1], 0.03333333333333333, Ops::mulc(f[0], 0.06666666666666667)))));
    b[7] = Ops::mul(vol, Ops::fmac(f[3], 0.03333333333333333, Ops::fmac(f[2], 0.06666666666666667, Ops::fmac(f[1], 0.06666666666666667, Ops::mulc(f[0], 0.03333333333333333)))));
    b[8] = Ops::mul(vol, Ops::fmac(f[3], 0.06666666666666667, Ops::fmac(f[2], 0.03333333333333333, Ops::fmac(f[1], 0.06666666666666667, Ops::mulc(f[0], 0.03333333333333333)))));
    b[9] = Ops::mul(vol, Ops::fmac(f[3], 0.06666666666666667, Ops::fmac(f[2], 0.06666666666666667, Ops::fmac(f[1], 0.03333333333333333, Ops::mulc(f[0], 0.03333333333333333)))));
  }
};

template <> struct Kappa<2, 1> {
  static constexpr int NKL = 18;
  // K[u] = sum_{k,(m<=n)} KL[k*NLAM + mn] * C[k][mn][i][j], KL = kappa_k * Lam_mn
  template <class Ops> __device__ __forceinline__ static void upper(const typename Ops::T* KL, typename Ops::T* K) {
    K[0] = Ops::fmac(KL[12], 0.3333333333333333, Ops::fmac(KL[6], 0.3333333333333333, Ops::mulc(KL[0], 0.3333333333333333)));
    K[1] = Ops::fmac(KL[13], 0.3333333333333333, Ops::fmac(KL[7], 0.3333333333333333, Ops::mulc(KL[1], 0.3333333333333333)));
    K[2] = Ops::fmac(KL[14], 0.3333333333333333, Ops::fmac(KL[8], 0.3333333333333333, Ops::mulc(KL[2], 0.3333333333333333)));
    K[3] = Ops::fmac(KL[15], 0.3333333333333333, Ops::fmac(KL[9], 0.3333333333333333, Ops::mulc(KL[3], 0.3333333333333333)));
    K[4] = Ops::fmac(KL[16], 0.3333333333333333, Ops::fmac(KL[10], 0.3333333333333333, Ops::mulc(KL[4], 0.3333333333333333)));
    K[5] = Ops::fmac(KL[17], 0.3333333333333333, Ops::fmac(KL[11], 0.3333333333333333, Ops::mulc(KL[5], 0.3333333333333333)));
  }
  static constexpr int TERMS = 18;
};

template <> struct Kappa<2, 2> {
  static constexpr int NKL = 18;
  // K[u] = sum_{k,(m<=n)} KL[k*NLAM + mn] * C[k][mn][i][j], KL = kappa_k * Lam_mn
  template <class Ops> __device__ __forceinline__ static void upper(const typename Ops::T* KL, typename Ops::T* K) {
    K[0] = Ops::fmac(KL[12], 0.2, Ops::fmac(KL[6], 0.2, Ops::mulc(KL[0], 0.6)));
    K[1] = Ops::fmac(KL[13], -0.06666666666666667, Ops::fmac(KL[7], -0.13333333333333333, Ops::mulc(KL[1], -0.13333333333333333)));
    K[2] = Ops::fmac(KL[14], -0.13333333333333333, Ops::fmac(KL[8], -0.06666666666666667, Ops::mulc(KL[2], -0.13333333333333333)));
    K[3] = Ops::fmac(KL[13], 0.2, Ops::fmac(KL[12], -0.06666666666666667, Ops::fmac(KL[7], 0.2, Ops::fmac(KL[6], -0.13333333333333333, Ops::fmac(KL[1], 0.9333333333333333, Ops::mulc(KL[0], 0.2))))));
    K[4] = Ops::fmac(KL[14], 0.2, Ops::fmac(KL[12], -0.13333333333333333, Ops::fmac(KL[8], 0.2, Ops::fmac(KL[6], -0.06666666666666667, Ops::fmac(KL[2], 0.9333333333333333, Ops::mulc(KL[0], 0.2))))));
    K[5] = Ops::fmac(KL[14], -0.06666666666666667, Ops::fmac(KL[13], -0.13333333333333333, Ops::fmac(KL[8], -0.13333333333333333, Ops::fmac(KL[7], -0.06666666666666667, Ops::fmac(KL[2], 0.2, Ops::mulc(KL[1], 0.2))))));
    K[6] = Ops::fmac(KL[15], 0.2, Ops::fmac(KL[9], 0.6, Ops::mulc(KL[3], 0.2)));
    K[7] = Ops::fmac(KL[16], -0.13333333333333333, Ops::fmac(KL[10], -0.13333333333333333, Ops::mulc(KL[4], -0.06666666666666667)));
    K[8] = Ops::fmac(KL[15], -0.06666666666666667, Ops::fmac(KL[13], 0.2, Ops::fmac(KL[9], 0.2, Ops::fmac(KL[7], 0.9333333333333333, Ops::fmac(KL[3], -0.13333333333333333, Ops::mulc(KL[1], 0.2))))));
    K[9] = Ops::fmac(KL[16], -0.06666666666666667, Ops::fmac(KL[13], -0.13333333333333333, Ops::fmac(KL[10], 0.2, Ops::fmac(KL[7], 0.2, Ops::fmac(KL[4], -0.13333333333333333, Ops::mulc(KL[1], -0.06666666666666667))))));
    K[10] = Ops::fmac(KL[16], 0.2, Ops::fmac(KL[15], -0.13333333333333333, Ops::fmac(KL[10], 0.9333333333333333, Ops::fmac(KL[9], 0.2, Ops::fmac(KL[4], 0.2, Ops::mulc(KL[3], -0.06666666666666667))))));
    K[11] = Ops::fmac(KL[17], 0.6, Ops::fmac(KL[11], 0.2, Ops::mulc(KL[5], 0.2)));
    K[12] = Ops::fmac(KL[16], 0.2, Ops::fmac(KL[14], 0.2, Ops::fmac(KL[10], -0.06666666666666667, Ops::fmac(KL[8], -0.13333333333333333, Ops::fmac(KL[4], -0.13333333333333333, Ops::mulc(KL[2], -0.06666666666666667))))));
    K[13] = Ops::fmac(KL[17], 0.2, Ops::fmac(KL[14], 0.9333333333333333, Ops::fmac(KL[11], -0.06666666666666667, Ops::fmac(KL[8], 0.2, Ops::fmac(KL[5], -0.13333333333333333, Ops::mulc(KL[2], 0.2))))));
    K[14] = Ops::fmac(KL[17], 0.2, Ops::fmac(KL[16], 0.9333333333333333, Ops::fmac(KL[11], -0.13333333333333333, Ops::fmac(KL[10], 0.2, Ops::fmac(KL[5], -0.06666666666666667, Ops::mulc(KL[4], 0.2))))));
    K[15] = Ops::fmac(KL[15], 0.5333333333333333, Ops::fmac(KL[13], 0.5333333333333333, Ops::fmac(KL[12], 0.5333333333333333, Ops::fmac(KL[9], 0.5333333333333333, Ops::fmac(KL[7], 1.0666666666666667, Ops::fmac(KL[6], 1.6, Ops::fmac(KL[3], 1.6, Ops::fmac(KL[1], 1.0666666666666667, Ops::mulc(KL[0], 0.5333333333333333)))))))));
    K[16] = Ops::fmac(KL[16], 0.5333333333333333, Ops::fmac(KL[14], 0.26666666666666666, Ops::fmac(KL[13], 0.5333333333333333, Ops::fmac(KL[12], 0.5333333333333333, Ops::fmac(KL[10], 0.5333333333333333, Ops::fmac(KL[8], 0.5333333333333333, Ops::fmac(KL[7], 0.26666666666666666, Ops::fmac(KL[6], 0.5333333333333333, Ops::fmac(KL[4], 1.6, Ops::fmac(KL[2], 0.5333333333333333, Ops::fmac(KL[1], 0.5333333333333333, Ops::mulc(KL[0], 0.26666666666666666))))))))))));
    K[17] = Ops::fmac(KL[16], 0.26666666666666666, Ops::fmac(KL[15], 0.5333333333333333, Ops::fmac(KL[14], 0.5333333333333333, Ops::fmac(KL[13], 0.5333333333333333, Ops::fmac(KL[10], 0.5333333333333333, Ops::fmac(KL[9], 0.26666666666666666, Ops::fmac(KL[8], 1.6, Ops::fmac(KL[7], 0.5333333333333333, Ops::fmac(KL[4], 0.5333333333333333, Ops::fmac(KL[3], 0.5333333333333333, Ops::fmac(KL[2], 0.5333333333333333, Ops::mulc(KL[1], 0.26666666666666666))))))))))));
    K[18] = Ops::fmac(KL[17], 0.5333333333333333, Ops::fmac(KL[14], 1.0666666666666667, Ops::fmac(KL[12], 1.6, Ops::fmac(KL[11], 0.5333333333333333, Ops::fmac(KL[8], 0.5333333333333333, Ops::fmac(KL[6], 0.5333333333333333, Ops::fmac(KL[5], 1.6, Ops::fmac(KL[2], 1.0666666666666667, Ops::mulc(KL[0], 0.5333333333333333)))))))));
    K[19] = Ops::fmac(KL[17], 0.26666666666666666, Ops::fmac(KL[16], 0.5333333333333333, Ops::fmac(KL[14], 0.5333333333333333, Ops::fmac(KL[13], 1.6, Ops::fmac(KL[11], 0.5333333333333333, Ops::fmac(KL[10], 0.26666666666666666, Ops::fmac(KL[8], 0.5333333333333333, Ops::fmac(KL[7], 0.5333333333333333, Ops::fmac(KL[5], 0.5333333333333333, Ops::fmac(KL[4], 0.5333333333333333, Ops::fmac(KL[2], 0.26666666666666666, Ops::mulc(KL[1], 0.5333333333333333))))))))))));
    K[20] = Ops::fmac(KL[17], 0.5333333333333333, Ops::fmac(KL[16], 1.0666666666666667, Ops::fmac(KL[15], 1.6, Ops::fmac(KL[11], 1.6, Ops::fmac(KL[10], 1.0666666666666667, Ops::fmac(KL[9], 0.5333333333333333, Ops::fmac(KL[5], 0.5333333333333333, Ops::fmac(KL[4], 0.5333333333333333, Ops::mulc(KL[3], 0.5333333333333333)))))))));
  }
  static constexpr int TERMS = 135;
};

template <> struct Kappa<2, 4> {
  static constexpr int NKL = 18;
  // K[u] = sum_{k,(m<=n)} KL[k*NLAM + mn] * C[k][mn][i][j], KL = kappa_k * Lam_mn
  template <class Ops> __device__ __forceinline__ static void upper(const typename Ops::T* KL, typename Ops::T* K) {
    K[0] = Ops::fmac(KL[12], 0.07583774250440917, Ops::fmac(KL[6], 0.07583774250440917, Ops::mulc(KL[0], 0.5943562610229277)));
    K[1] = Ops::fmac(KL[13], -0.010229276895943563, Ops::fmac(KL[7], -0.051499118165784834, Ops::mulc(KL[1], -0.051499118165784834)));
    K[2] = Ops::fmac(KL[14], -0.051499118165784834, Ops::fmac(KL[8], -0.010229276895943563, Ops::mulc(KL[2], -0.051499118165784834)));
    K[3] = Ops::fmac(KL[13], 0.09171075837742504, Ops::fmac(KL[12], -0.04938271604938271, Ops::fmac(KL[7], 0.09171075837742504, Ops::fmac(KL[6], -0.09876543209876543, Ops::fmac(KL[1], 1.3742504409171077, Ops::mulc(KL[0], 0.4021164021164021))))));
    K[4] = Ops::fmac(KL[13], -0.06525573192239859, Ops::fmac(KL[12], 0.04056437389770723, Ops::fmac(KL[7], -0.05114638447971781, Ops::fmac(KL[6], 0.17989417989417988, Ops::fmac(KL[1], -0.7343915343915344, Ops::mulc(KL[0], -0.13580246913580246))))));
    K[5] = Ops::fmac(KL[13], 0.03527336860670194, Ops::fmac(KL[12], -0.015520282186948854, Ops::fmac(KL[7], 0.06349206349206349, Ops::fmac(KL[6], -0.10440917107583775, Ops::fmac(KL[1], 0.3075837742504409, Ops::mulc(KL[0], 0.03527336860670194))))));
    K[6] = Ops::fmac(KL[14], 0.09171075837742504, Ops::fmac(KL[12], -0.09876543209876543, Ops::fmac(KL[8], 0.09171075837742504, Ops::fmac(KL[6], -0.04938271604938271, Ops::fmac(KL[2], 1.3742504409171077, Ops::mulc(KL[0], 0.4021164021164021))))));
    K[7] = Ops::fmac(KL[14], -0.05114638447971781, Ops::fmac(KL[12], 0.17989417989417988, Ops::fmac(KL[8], -0.06525573192239859, Ops::fmac(KL[6], 0.04056437389770723, Ops::fmac(KL[2], -0.7343915343915344, Ops::mulc(KL[0], -0.13580246913580246))))));
    K[8] = Ops::fmac(KL[14], 0.06349206349206349, Ops::fmac(KL[12], -0.10440917107583775, Ops::fmac(KL[8], 0.03527336860670194, Ops::fmac(KL[6], -0.015520282186948854, Ops::fmac(KL[2], 0.3075837742504409, Ops::mulc(KL[0], 0.03527336860670194))))));
    K[9] = Ops::fmac(KL[14], -0.015520282186948854, Ops::fmac(KL[13], -0.031040564373897708, Ops::fmac(KL[8], -0.10440917107583775, Ops::fmac(KL[7], -0.08888888888888889, Ops::fmac(KL[2], 0.03527336860670194, Ops::mulc(KL[1], 0.03527336860670194))))));
    K[10] = Ops::fmac(KL[14], -0.04691358024691358, Ops::fmac(KL[13], -0.05714285714285714, Ops::fmac(KL[8], -0.05714285714285714, Ops::fmac(KL[7], -0.04691358024691358, Ops::fmac(KL[2], 0.019400352733686066, Ops::mulc(KL[1], 0.019400352733686066))))));
    K[11] = Ops::fmac(KL[14], -0.08888888888888889, Ops::fmac(KL[13], -0.10440917107583775, Ops::fmac(KL[8], -0.031040564373897708, Ops::fmac(KL[7], -0.015520282186948854, Ops::fmac(KL[2], 0.03527336860670194, Ops::mulc(KL[1], 0.03527336860670194))))));
    K[12] = Ops::fmac(KL[14], 0.014109347442680775, Ops::fmac(KL[13], 0.02821869488536155, Ops::fmac(KL[12], 0.19753086419753085, Ops::fmac(KL[8], 0.02821869488536155, Ops::fmac(KL[7], 0.014109347442680775, Ops::fmac(KL[6], 0.19753086419753085, Ops::fmac(KL[2], 0.5925925925925926, Ops::fmac(KL[1], 0.5925925925925926, Ops::mulc(KL[0], 0.07054673721340388)))))))));
    K[13] = Ops::fmac(KL[14], 0.014109347442680775, Ops::fmac(KL[13], 0.02821869488536155, Ops::fmac(KL[12], -0.07336860670194004, Ops::fmac(KL[8], 0.08465608465608465, Ops::fmac(KL[7], 0.07054673721340388, Ops::fmac(KL[6], -0.1523809523809524, Ops::fmac(KL[2], -0.14109347442680775, Ops::fmac(KL[1], -0.14109347442680775, Ops::mulc(KL[0], 0.014109347442680775)))))))));
    K[14] = Ops::fmac(KL[14], 0.07054673721340388, Ops::fmac(KL[13], 0.08465608465608465, Ops::fmac(KL[12], -0.1523809523809524, Ops::fmac(KL[8], 0.02821869488536155, Ops::fmac(KL[7], 0.014109347442680775, Ops::fmac(KL[6], -0.07336860670194004, Ops::fmac(KL[2], -0.14109347442680775, Ops::fmac(KL[1], -0.14109347442680775, Ops::mulc(KL[0], 0.014109347442680775)))))))));
    K[15] = Ops::fmac(KL[15], 0.07583774250440917, Ops::fmac(KL[9], 0.5943562610229277, Ops::mulc(KL[3], 0.07583774250440917)));
    K[16] = Ops::fmac(KL[16], -0.051499118165784834, Ops::fmac(KL[10], -0.051499118165784834, Ops::mulc(KL[4], -0.010229276895943563)));
    K[17] = Ops::fmac(KL[15], -0.015520282186948854, Ops::fmac(KL[13], 0.03527336860670194, Ops::fmac(KL[9], 0.03527336860670194, Ops::fmac(KL[7], 0.3075837742504409, Ops::fmac(KL[3], -0.10440917107583775, Ops::mulc(KL[1], 0.06349206349206349))))));
    K[18] = Ops::fmac(KL[15], 0.04056437389770723, Ops::fmac(KL[13], -0.06525573192239859, Ops::fmac(KL[9], -0.13580246913580246, Ops::fmac(KL[7], -0.7343915343915344, Ops::fmac(KL[3], 0.17989417989417988, Ops::mulc(KL[1], -0.05114638447971781))))));
    K[19] = Ops::fmac(KL[15], -0.04938271604938271, Ops::fmac(KL[13], 0.09171075837742504, Ops::fmac(KL[9], 0.4021164021164021, Ops::fmac(KL[7], 1.3742504409171077, Ops::fmac(KL[3], -0.09876543209876543, Ops::mulc(KL[1], 0.09171075837742504))))));
    K[20] = Ops::fmac(KL[16], -0.015520282186948854, Ops::fmac(KL[13], -0.031040564373897708, Ops::fmac(KL[10], 0.03527336860670194, Ops::fmac(KL[7], 0.03527336860670194, Ops::fmac(KL[4], -0.10440917107583775, Ops::mulc(KL[1], -0.08888888888888889))))));
    K[21] = Ops::fmac(KL[16], -0.04691358024691358, Ops::fmac(KL[13], -0.05714285714285714, Ops::fmac(KL[10], 0.019400352733686066, Ops::fmac(KL[7], 0.019400352733686066, Ops::fmac(KL[4], -0.05714285714285714, Ops::mulc(KL[1], -0.04691358024691358))))));
    K[22] = Ops::fmac(KL[16], -0.08888888888888889, Ops::fmac(KL[13], -0.10440917107583775, Ops::fmac(KL[10], 0.03527336860670194, Ops::fmac(KL[7], 0.03527336860670194, Ops::fmac(KL[4], -0.031040564373897708, Ops::mulc(KL[1], -0.015520282186948854))))));
    K[23] = Ops::fmac(KL[16], 0.09171075837742504, Ops::fmac(KL[15], -0.09876543209876543, Ops::fmac(KL[10], 1.3742504409171077, Ops::fmac(KL[9], 0.4021164021164021, Ops::fmac(KL[4], 0.09171075837742504, Ops::mulc(KL[3], -0.04938271604938271))))));
    K[24] = Ops::fmac(KL[16], -0.05114638447971781, Ops::fmac(KL[15], 0.17989417989417988, Ops::fmac(KL[10], -0.7343915343915344, Ops::fmac(KL[9], -0.13580246913580246, Ops::fmac(KL[4], -0.06525573192239859, Ops::mulc(KL[3], 0.04056437389770723))))));
    K[25] = Ops::fmac(KL[16], 0.06349206349206349, Ops::fmac(KL[15], -0.10440917107583775, Ops::fmac(KL[10], 0.3075837742504409, Ops::fmac(KL[9], 0.03527336860670194, Ops::fmac(KL[4], 0.03527336860670194, Ops::mulc(KL[3], -0.015520282186948854))))));
    K[26] = Ops::fmac(KL[16], 0.014109347442680775, Ops::fmac(KL[15], -0.07336860670194004, Ops::fmac(KL[13], 0.02821869488536155, Ops::fmac(KL[10], -0.14109347442680775, Ops::fmac(KL[9], 0.014109347442680775, Ops::fmac(KL[7], -0.14109347442680775, Ops::fmac(KL[4], 0.08465608465608465, Ops::fmac(KL[3], -0.1523809523809524, Ops::mulc(KL[1], 0.07054673721340388)))))))));
    K[27] = Ops::fmac(KL[16], 0.014109347442680775, Ops::fmac(KL[15], 0.19753086419753085, Ops::fmac(KL[13], 0.02821869488536155, Ops::fmac(KL[10], 0.5925925925925926, Ops::fmac(KL[9], 0.07054673721340388, Ops::fmac(KL[7], 0.5925925925925926, Ops::fmac(KL[4], 0.02821869488536155, Ops::fmac(KL[3], 0.19753086419753085, Ops::mulc(KL[1], 0.014109347442680775)))))))));
    K[28] = Ops::fmac(KL[16], 0.07054673721340388, Ops::fmac(KL[15], -0.1523809523809524, Ops::fmac(KL[13], 0.08465608465608465, Ops::fmac(KL[10], -0.14109347442680775, Ops::fmac(KL[9], 0.014109347442680775, Ops::fmac(KL[7], -0.14109347442680775, Ops::fmac(KL[4], 0.02821869488536155, Ops::fmac(KL[3], -0.07336860670194004, Ops::mulc(KL[1], 0.014109347442680775)))))))));
    K[29] = Ops::fmac(KL[17], 0.5943562610229277, Ops::fmac(KL[11], 0.07583774250440917, Ops::mulc(KL[5], 0.07583774250440917)));
    K[30] = Ops::fmac(KL[16], 0.03527336860670194, Ops::fmac(KL[14], 0.03527336860670194, Ops::fmac(KL[10], -0.015520282186948854, Ops::fmac(KL[8], -0.031040564373897708, Ops::fmac(KL[4], -0.10440917107583775, Ops::mulc(KL[2], -0.08888888888888889))))));
    K[31] = Ops::fmac(KL[16], 0.019400352733686066, Ops::fmac(KL[14], 0.019400352733686066, Ops::fmac(KL[10], -0.04691358024691358, Ops::fmac(KL[8], -0.05714285714285714, Ops::fmac(KL[4], -0.05714285714285714, Ops::mulc(KL[2], -0.04691358024691358))))));
    K[32] = Ops::fmac(KL[16], 0.03527336860670194, Ops::fmac(KL[14], 0.03527336860670194, Ops::fmac(KL[10], -0.08888888888888889, Ops::fmac(KL[8], -0.10440917107583775, Ops::fmac(KL[4], -0.031040564373897708, Ops::mulc(KL[2], -0.015520282186948854))))));
    K[33] = Ops::fmac(KL[17], 0.03527336860670194, Ops::fmac(KL[14], 0.3075837742504409, Ops::fmac(KL[11], -0.015520282186948854, Ops::fmac(KL[8], 0.03527336860670194, Ops::fmac(KL[5], -0.10440917107583775, Ops::mulc(KL[2], 0.06349206349206349))))));
    K[34] = Ops::fmac(KL[17], -0.13580246913580246, Ops::fmac(KL[14], -0.7343915343915344, Ops::fmac(KL[11], 0.04056437389770723, Ops::fmac(KL[8], -0.06525573192239859, Ops::fmac(KL[5], 0.17989417989417988, Ops::mulc(KL[2], -0.05114638447971781))))));
    K[35] = Ops::fmac(KL[17], 0.4021164021164021, Ops::fmac(KL[14], 1.3742504409171077, Ops::fmac(KL[11], -0.04938271604938271, Ops::fmac(KL[8], 0.09171075837742504, Ops::fmac(KL[5], -0.09876543209876543, Ops::mulc(KL[2], 0.09171075837742504))))));
    K[36] = Ops::fmac(KL[17], 0.03527336860670194, Ops::fmac(KL[16], 0.3075837742504409, Ops::fmac(KL[11], -0.10440917107583775, Ops::fmac(KL[10], 0.06349206349206349, Ops::fmac(KL[5], -0.015520282186948854, Ops::mulc(KL[4], 0.03527336860670194))))));
    K[37] = Ops::fmac(KL[17], -0.13580246913580246, Ops::fmac(KL[16], -0.7343915343915344, Ops::fmac(KL[11], 0.17989417989417988, Ops::fmac(KL[10], -0.05114638447971781, Ops::fmac(KL[5], 0.04056437389770723, Ops::mulc(KL[4], -0.06525573192239859))))));
    K[38] = Ops::fmac(KL[17], 0.4021164021164021, Ops::fmac(KL[16], 1.3742504409171077, Ops::fmac(KL[11], -0.09876543209876543, Ops::fmac(KL[10], 0.09171075837742504, Ops::fmac(KL[5], -0.04938271604938271, Ops::mulc(KL[4], 0.09171075837742504))))));
    K[39] = Ops::fmac(KL[17], 0.014109347442680775, Ops::fmac(KL[16], -0.14109347442680775, Ops::fmac(KL[14], -0.14109347442680775, Ops::fmac(KL[11], -0.07336860670194004, Ops::fmac(KL[10], 0.014109347442680775, Ops::fmac(KL[8], 0.02821869488536155, Ops::fmac(KL[5], -0.1523809523809524, Ops::fmac(KL[4], 0.08465608465608465, Ops::mulc(KL[2], 0.07054673721340388)))))))));
    K[40] = Ops::fmac(KL[17], 0.014109347442680775, Ops::fmac(KL[16], -0.14109347442680775, Ops::fmac(KL[14], -0.14109347442680775, Ops::fmac(KL[11], -0.1523809523809524, Ops::fmac(KL[10], 0.07054673721340388, Ops::fmac(KL[8], 0.08465608465608465, Ops::fmac(KL[5], -0.07336860670194004, Ops::fmac(KL[4], 0.02821869488536155, Ops::mulc(KL[2], 0.014109347442680775)))))))));
    K[41] = Ops::fmac(KL[17], 0.07054673721340388, Ops::fmac(KL[16], 0.5925925925925926, Ops::fmac(KL[14], 0.5925925925925926, Ops::fmac(KL[11], 0.19753086419753085, Ops::fmac(KL[10], 0.014109347442680775, Ops::fmac(KL[8], 0.02821869488536155, Ops::fmac(KL[5], 0.19753086419753085, Ops::fmac(KL[4], 0.02821869488536155, Ops::mulc(KL[2], 0.014109347442680775)))))))));
    K[42] = Ops::fmac(KL[15], 0.3160493827160494, Ops::fmac(KL[13], 0.3160493827160494, Ops::fmac(KL[12], 0.40634920634920635, Ops::fmac(KL[9], 0.3160493827160494, Ops::fmac(KL[7], 0.6320987654320988, Ops::fmac(KL[6], 1.2190476190476192, Ops::fmac(KL[3], 3.5668430335097003, Ops::fmac(KL[1], 3.250793650793651, Ops::mulc(KL[0], 2.0317460317460316)))))))));
    K[43] = Ops::fmac(KL[15], -0.18059964726631395, Ops::fmac(KL[13], 0.022574955908289243, Ops::fmac(KL[12], -0.23703703703703705, Ops::fmac(KL[9], 0.045149911816578486, Ops::fmac(KL[7], 0.4740740740740741, Ops::fmac(KL[6], -0.9142857142857143, Ops::fmac(KL[3], -1.3883597883597885, Ops::fmac(KL[1], 0.5530864197530864, Ops::mulc(KL[0], -0.1693121693121693)))))))));
    K[44] = Ops::fmac(KL[15], 0.09029982363315697, Ops::fmac(KL[13], -0.045149911816578486, Ops::fmac(KL[12], 0.09029982363315697, Ops::fmac(KL[7], -0.3160493827160494, Ops::fmac(KL[6], 0.5869488536155203, Ops::fmac(KL[3], 0.5869488536155203, Ops::mulc(KL[1], -0.3160493827160494)))))));
    K[45] = Ops::fmac(KL[16], 0.3160493827160494, Ops::fmac(KL[14], 0.1580246913580247, Ops::fmac(KL[13], 0.3160493827160494, Ops::fmac(KL[12], 0.40634920634920635, Ops::fmac(KL[10], 0.3160493827160494, Ops::fmac(KL[8], 0.3160493827160494, Ops::fmac(KL[7], 0.1580246913580247, Ops::fmac(KL[6], 0.40634920634920635, Ops::fmac(KL[4], 3.5668430335097003, Ops::fmac(KL[2], 1.6253968253968254, Ops::fmac(KL[1], 1.6253968253968254, Ops::mulc(KL[0], 1.0158730158730158))))))))))));
    K[46] = Ops::fmac(KL[16], 0.045149911816578486, Ops::fmac(KL[14], 0.08465608465608465, Ops::fmac(KL[13], -0.10158730158730159, Ops::fmac(KL[12], -0.23703703703703705, Ops::fmac(KL[10], -0.18059964726631395, Ops::fmac(KL[8], -0.23703703703703705, Ops::fmac(KL[7], -0.062081128747795415, Ops::fmac(KL[6], -0.1693121693121693, Ops::fmac(KL[4], -1.3883597883597885, Ops::fmac(KL[2], -0.7788359788359789, Ops::fmac(KL[1], -0.4289241622574956, Ops::mulc(KL[0], -0.3216931216931217))))))))))));
    K[47] = Ops::fmac(KL[14], -0.06772486772486773, Ops::fmac(KL[13], 0.09029982363315697, Ops::fmac(KL[12], 0.09029982363315697, Ops::fmac(KL[10], 0.09029982363315697, Ops::fmac(KL[8], 0.13544973544973546, Ops::fmac(KL[7], 0.022574955908289243, Ops::fmac(KL[6], 0.045149911816578486, Ops::fmac(KL[4], 0.5869488536155203, Ops::fmac(KL[2], 0.40634920634920635, Ops::fmac(KL[1], 0.09029982363315697, Ops::mulc(KL[0], 0.06772486772486773)))))))))));
    K[48] = Ops::fmac(KL[16], 0.022574955908289243, Ops::fmac(KL[15], 0.045149911816578486, Ops::fmac(KL[14], 0.09029982363315697, Ops::fmac(KL[13], 0.13544973544973546, Ops::fmac(KL[10], 0.09029982363315697, Ops::fmac(KL[9], 0.06772486772486773, Ops::fmac(KL[8], 0.5869488536155203, Ops::fmac(KL[7], 0.40634920634920635, Ops::fmac(KL[4], 0.09029982363315697, Ops::fmac(KL[3], 0.09029982363315697, Ops::mulc(KL[1], -0.06772486772486773)))))))))));
    K[49] = Ops::fmac(KL[16], 0.02821869488536155, Ops::fmac(KL[15], 0.033862433862433865, Ops::fmac(KL[14], 0.1693121693121693, Ops::fmac(KL[13], 0.1693121693121693, Ops::fmac(KL[10], 0.033862433862433865, Ops::fmac(KL[9], 0.02821869488536155, Ops::fmac(KL[8], 0.1693121693121693, Ops::fmac(KL[7], 0.10158730158730159, Ops::fmac(KL[4], 0.022574955908289243, Ops::fmac(KL[3], 0.022574955908289243, Ops::fmac(KL[2], -0.033862433862433865, Ops::mulc(KL[1], -0.050793650793650794))))))))))));
    K[50] = Ops::fmac(KL[16], 0.06772486772486773, Ops::fmac(KL[15], 0.09029982363315697, Ops::fmac(KL[14], 0.13544973544973546, Ops::fmac(KL[13], 0.09029982363315697, Ops::fmac(KL[10], 0.045149911816578486, Ops::fmac(KL[9], 0.022574955908289243, Ops::fmac(KL[8], 0.13544973544973546, Ops::fmac(KL[7], 0.045149911816578486, Ops::fmac(KL[4], 0.09029982363315697, Ops::fmac(KL[3], 0.09029982363315697, Ops::fmac(KL[2], 0.13544973544973546, Ops::mulc(KL[1], 0.06772486772486773))))))))))));
    K[51] = Ops::fmac(KL[16], 0.2257495590828924, Ops::fmac(KL[15], 0.4514991181657848, Ops::fmac(KL[14], 0.40634920634920635, Ops::fmac(KL[13], 0.4514991181657848, Ops::fmac(KL[12], -0.2708994708994709, Ops::fmac(KL[10], 0.4514991181657848, Ops::fmac(KL[9], 0.2257495590828924, Ops::fmac(KL[8], 1.2190476190476192, Ops::fmac(KL[7], 0.4514991181657848, Ops::fmac(KL[6], -0.40634920634920635, Ops::fmac(KL[4], 2.5735449735449736, Ops::fmac(KL[3], 2.5735449735449736, Ops::fmac(KL[2], 3.5216931216931218, Ops::fmac(KL[1], 2.347795414462081, Ops::mulc(KL[0], 0.9481481481481482)))))))))))))));
    K[52] = Ops::fmac(KL[16], -0.045149911816578486, Ops::fmac(KL[15], -0.09029982363315697, Ops::fmac(KL[14], -0.13544973544973546, Ops::fmac(KL[13], -0.09029982363315697, Ops::fmac(KL[12], 0.2708994708994709, Ops::fmac(KL[9], 0.045149911816578486, Ops::fmac(KL[8], -0.40634920634920635, Ops::fmac(KL[6], 0.6772486772486772, Ops::fmac(KL[4], -0.4966490299823633, Ops::fmac(KL[3], -0.4966490299823633, Ops::fmac(KL[2], -0.2708994708994709, Ops::fmac(KL[1], 0.09029982363315697, Ops::mulc(KL[0], -0.13544973544973546)))))))))))));
    K[53] = Ops::fmac(KL[16], 0.045149911816578486, Ops::fmac(KL[14], -0.13544973544973546, Ops::fmac(KL[12], 0.2708994708994709, Ops::fmac(KL[10], -0.09029982363315697, Ops::fmac(KL[9], -0.045149911816578486, Ops::fmac(KL[8], -0.40634920634920635, Ops::fmac(KL[7], -0.09029982363315697, Ops::fmac(KL[6], 0.13544973544973546, Ops::fmac(KL[4], -0.4966490299823633, Ops::fmac(KL[3], -0.4966490299823633, Ops::fmac(KL[2], -0.8126984126984127, Ops::fmac(KL[1], -0.4514991181657848, Ops::mulc(KL[0], -0.13544973544973546)))))))))))));
    K[54] = Ops::fmac(KL[15], 0.49947089947089945, Ops::fmac(KL[13], 0.33015873015873015, Ops::fmac(KL[12], 0.49947089947089945, Ops::fmac(KL[9], 1.2444444444444445, Ops::fmac(KL[7], 1.7777777777777777, Ops::fmac(KL[6], 3.157671957671958, Ops::fmac(KL[3], 3.157671957671958, Ops::fmac(KL[1], 1.7777777777777777, Ops::mulc(KL[0], 1.2444444444444445)))))))));
    K[55] = Ops::fmac(KL[15], -0.23703703703703705, Ops::fmac(KL[13], 0.022574955908289243, Ops::fmac(KL[12], -0.18059964726631395, Ops::fmac(KL[9], -0.1693121693121693, Ops::fmac(KL[7], 0.5530864197530864, Ops::fmac(KL[6], -1.3883597883597885, Ops::fmac(KL[3], -0.9142857142857143, Ops::fmac(KL[1], 0.4740740740740741, Ops::mulc(KL[0], 0.045149911816578486)))))))));
    K[56] = Ops::fmac(KL[16], -0.18059964726631395, Ops::fmac(KL[14], -0.062081128747795415, Ops::fmac(KL[13], -0.23703703703703705, Ops::fmac(KL[12], -0.1693121693121693, Ops::fmac(KL[10], 0.045149911816578486, Ops::fmac(KL[8], -0.10158730158730159, Ops::fmac(KL[7], 0.08465608465608465, Ops::fmac(KL[6], -0.23703703703703705, Ops::fmac(KL[4], -1.3883597883597885, Ops::fmac(KL[2], -0.4289241622574956, Ops::fmac(KL[1], -0.7788359788359789, Ops::mulc(KL[0], -0.3216931216931217))))))))))));
    K[57] = Ops::fmac(KL[16], -0.21164021164021163, Ops::fmac(KL[14], -0.10582010582010581, Ops::fmac(KL[13], -0.12698412698412698, Ops::fmac(KL[12], -0.09312169312169312, Ops::fmac(KL[10], -0.21164021164021163, Ops::fmac(KL[8], -0.12698412698412698, Ops::fmac(KL[7], -0.10582010582010581, Ops::fmac(KL[6], -0.09312169312169312, Ops::fmac(KL[4], -0.364021164021164, Ops::fmac(KL[2], -0.16084656084656085, Ops::fmac(KL[1], -0.16084656084656085, Ops::mulc(KL[0], -0.10582010582010581))))))))))));
    K[58] = Ops::fmac(KL[16], -0.033862433862433865, Ops::fmac(KL[14], -0.050793650793650794, Ops::fmac(KL[13], 0.022574955908289243, Ops::fmac(KL[12], 0.022574955908289243, Ops::fmac(KL[10], 0.1693121693121693, Ops::fmac(KL[8], 0.1693121693121693, Ops::fmac(KL[7], 0.02821869488536155, Ops::fmac(KL[6], 0.033862433862433865, Ops::fmac(KL[4], 0.1693121693121693, Ops::fmac(KL[2], 0.10158730158730159, Ops::fmac(KL[1], 0.033862433862433865, Ops::mulc(KL[0], 0.02821869488536155))))))))))));
    K[59] = Ops::fmac(KL[16], -0.062081128747795415, Ops::fmac(KL[15], -0.1693121693121693, Ops::fmac(KL[14], -0.18059964726631395, Ops::fmac(KL[13], -0.23703703703703705, Ops::fmac(KL[10], -0.4289241622574956, Ops::fmac(KL[9], -0.3216931216931217, Ops::fmac(KL[8], -1.3883597883597885, Ops::fmac(KL[7], -0.7788359788359789, Ops::fmac(KL[4], -0.10158730158730159, Ops::fmac(KL[3], -0.23703703703703705, Ops::fmac(KL[2], 0.045149911816578486, Ops::mulc(KL[1], 0.08465608465608465))))))))))));
    K[60] = Ops::fmac(KL[16], -0.10582010582010581, Ops::fmac(KL[15], -0.09312169312169312, Ops::fmac(KL[14], -0.21164021164021163, Ops::fmac(KL[13], -0.12698412698412698, Ops::fmac(KL[10], -0.16084656084656085, Ops::fmac(KL[9], -0.10582010582010581, Ops::fmac(KL[8], -0.364021164021164, Ops::fmac(KL[7], -0.16084656084656085, Ops::fmac(KL[4], -0.12698412698412698, Ops::fmac(KL[3], -0.09312169312169312, Ops::fmac(KL[2], -0.21164021164021163, Ops::mulc(KL[1], -0.10582010582010581))))))))))));
    K[61] = Ops::fmac(KL[16], -0.050793650793650794, Ops::fmac(KL[15], 0.022574955908289243, Ops::fmac(KL[14], -0.033862433862433865, Ops::fmac(KL[13], 0.022574955908289243, Ops::fmac(KL[10], 0.10158730158730159, Ops::fmac(KL[9], 0.02821869488536155, Ops::fmac(KL[8], 0.1693121693121693, Ops::fmac(KL[7], 0.033862433862433865, Ops::fmac(KL[4], 0.1693121693121693, Ops::fmac(KL[3], 0.033862433862433865, Ops::fmac(KL[2], 0.1693121693121693, Ops::mulc(KL[1], 0.02821869488536155))))))))))));
    K[62] = Ops::fmac(KL[16], 0.3724867724867725, Ops::fmac(KL[15], -0.3386243386243386, Ops::fmac(KL[14], 0.10158730158730159, Ops::fmac(KL[13], 0.20317460317460317, Ops::fmac(KL[12], 0.4740740740740741, Ops::fmac(KL[10], 1.8285714285714285, Ops::fmac(KL[9], 0.3724867724867725, Ops::fmac(KL[8], 1.1174603174603175, Ops::fmac(KL[7], 1.0158730158730158, Ops::fmac(KL[6], 1.6592592592592592, Ops::fmac(KL[4], 2.471957671957672, Ops::fmac(KL[3], -1.0497354497354496, Ops::fmac(KL[2], 0.6095238095238096, Ops::fmac(KL[1], 0.6095238095238096, Ops::mulc(KL[0], 0.5079365079365079)))))))))))))));
    K[63] = Ops::fmac(KL[16], 0.10158730158730159, Ops::fmac(KL[15], 0.4740740740740741, Ops::fmac(KL[14], 0.3724867724867725, Ops::fmac(KL[13], 0.20317460317460317, Ops::fmac(KL[12], -0.3386243386243386, Ops::fmac(KL[10], 0.6095238095238096, Ops::fmac(KL[9], 0.5079365079365079, Ops::fmac(KL[8], 2.471957671957672, Ops::fmac(KL[7], 0.6095238095238096, Ops::fmac(KL[6], -1.0497354497354496, Ops::fmac(KL[4], 1.1174603174603175, Ops::fmac(KL[3], 1.6592592592592592, Ops::fmac(KL[2], 1.8285714285714285, Ops::fmac(KL[1], 1.0158730158730158, Ops::mulc(KL[0], 0.3724867724867725)))))))))))))));
    K[64] = Ops::fmac(KL[16], -0.033862433862433865, Ops::fmac(KL[15], -0.20317460317460317, Ops::fmac(KL[14], -0.033862433862433865, Ops::fmac(KL[13], -0.3386243386243386, Ops::fmac(KL[12], -0.20317460317460317, Ops::fmac(KL[10], -0.6095238095238096, Ops::fmac(KL[9], -0.1693121693121693, Ops::fmac(KL[8], -0.7788359788359789, Ops::fmac(KL[7], -0.3386243386243386, Ops::fmac(KL[6], -0.23703703703703705, Ops::fmac(KL[4], -0.7788359788359789, Ops::fmac(KL[3], -0.23703703703703705, Ops::fmac(KL[2], -0.6095238095238096, Ops::fmac(KL[1], -0.3386243386243386, Ops::mulc(KL[0], -0.1693121693121693)))))))))))))));
    K[65] = Ops::fmac(KL[15], 0.40634920634920635, Ops::fmac(KL[13], 0.3160493827160494, Ops::fmac(KL[12], 0.3160493827160494, Ops::fmac(KL[9], 2.0317460317460316, Ops::fmac(KL[7], 3.250793650793651, Ops::fmac(KL[6], 3.5668430335097003, Ops::fmac(KL[3], 1.2190476190476192, Ops::fmac(KL[1], 0.6320987654320988, Ops::mulc(KL[0], 0.3160493827160494)))))))));
    K[66] = Ops::fmac(KL[16], 0.09029982363315697, Ops::fmac(KL[14], 0.022574955908289243, Ops::fmac(KL[13], 0.13544973544973546, Ops::fmac(KL[12], 0.045149911816578486, Ops::fmac(KL[8], 0.09029982363315697, Ops::fmac(KL[7], -0.06772486772486773, Ops::fmac(KL[6], 0.09029982363315697, Ops::fmac(KL[4], 0.5869488536155203, Ops::fmac(KL[2], 0.09029982363315697, Ops::fmac(KL[1], 0.40634920634920635, Ops::mulc(KL[0], 0.06772486772486773)))))))))));
    K[67] = Ops::fmac(KL[16], 0.1693121693121693, Ops::fmac(KL[14], 0.02821869488536155, Ops::fmac(KL[13], 0.1693121693121693, Ops::fmac(KL[12], 0.033862433862433865, Ops::fmac(KL[10], -0.033862433862433865, Ops::fmac(KL[8], 0.022574955908289243, Ops::fmac(KL[7], -0.050793650793650794, Ops::fmac(KL[6], 0.022574955908289243, Ops::fmac(KL[4], 0.1693121693121693, Ops::fmac(KL[2], 0.033862433862433865, Ops::fmac(KL[1], 0.10158730158730159, Ops::mulc(KL[0], 0.02821869488536155))))))))))));
    K[68] = Ops::fmac(KL[16], 0.13544973544973546, Ops::fmac(KL[14], 0.06772486772486773, Ops::fmac(KL[13], 0.09029982363315697, Ops::fmac(KL[12], 0.09029982363315697, Ops::fmac(KL[10], 0.13544973544973546, Ops::fmac(KL[8], 0.09029982363315697, Ops::fmac(KL[7], 0.06772486772486773, Ops::fmac(KL[6], 0.09029982363315697, Ops::fmac(KL[4], 0.13544973544973546, Ops::fmac(KL[2], 0.045149911816578486, Ops::fmac(KL[1], 0.045149911816578486, Ops::mulc(KL[0], 0.022574955908289243))))))))))));
    K[69] = Ops::fmac(KL[16], 0.1580246913580247, Ops::fmac(KL[15], 0.40634920634920635, Ops::fmac(KL[14], 0.3160493827160494, Ops::fmac(KL[13], 0.3160493827160494, Ops::fmac(KL[10], 1.6253968253968254, Ops::fmac(KL[9], 1.0158730158730158, Ops::fmac(KL[8], 3.5668430335097003, Ops::fmac(KL[7], 1.6253968253968254, Ops::fmac(KL[4], 0.3160493827160494, Ops::fmac(KL[3], 0.40634920634920635, Ops::fmac(KL[2], 0.3160493827160494, Ops::mulc(KL[1], 0.1580246913580247))))))))))));
    K[70] = Ops::fmac(KL[16], 0.08465608465608465, Ops::fmac(KL[15], -0.23703703703703705, Ops::fmac(KL[14], 0.045149911816578486, Ops::fmac(KL[13], -0.10158730158730159, Ops::fmac(KL[10], -0.7788359788359789, Ops::fmac(KL[9], -0.3216931216931217, Ops::fmac(KL[8], -1.3883597883597885, Ops::fmac(KL[7], -0.4289241622574956, Ops::fmac(KL[4], -0.23703703703703705, Ops::fmac(KL[3], -0.1693121693121693, Ops::fmac(KL[2], -0.18059964726631395, Ops::mulc(KL[1], -0.062081128747795415))))))))))));
    K[71] = Ops::fmac(KL[16], -0.06772486772486773, Ops::fmac(KL[15], 0.09029982363315697, Ops::fmac(KL[13], 0.09029982363315697, Ops::fmac(KL[10], 0.40634920634920635, Ops::fmac(KL[9], 0.06772486772486773, Ops::fmac(KL[8], 0.5869488536155203, Ops::fmac(KL[7], 0.09029982363315697, Ops::fmac(KL[4], 0.13544973544973546, Ops::fmac(KL[3], 0.045149911816578486, Ops::fmac(KL[2], 0.09029982363315697, Ops::mulc(KL[1], 0.022574955908289243)))))))))));
    K[72] = Ops::fmac(KL[16], -0.13544973544973546, Ops::fmac(KL[15], 0.2708994708994709, Ops::fmac(KL[14], -0.045149911816578486, Ops::fmac(KL[13], -0.09029982363315697, Ops::fmac(KL[12], -0.09029982363315697, Ops::fmac(KL[10], -0.2708994708994709, Ops::fmac(KL[9], -0.13544973544973546, Ops::fmac(KL[8], -0.4966490299823633, Ops::fmac(KL[7], 0.09029982363315697, Ops::fmac(KL[6], -0.4966490299823633, Ops::fmac(KL[4], -0.40634920634920635, Ops::fmac(KL[3], 0.6772486772486772, Ops::mulc(KL[0], 0.045149911816578486)))))))))))));
    K[73] = Ops::fmac(KL[16], 0.40634920634920635, Ops::fmac(KL[15], -0.2708994708994709, Ops::fmac(KL[14], 0.2257495590828924, Ops::fmac(KL[13], 0.4514991181657848, Ops::fmac(KL[12], 0.4514991181657848, Ops::fmac(KL[10], 3.5216931216931218, Ops::fmac(KL[9], 0.9481481481481482, Ops::fmac(KL[8], 2.5735449735449736, Ops::fmac(KL[7], 2.347795414462081, Ops::fmac(KL[6], 2.5735449735449736, Ops::fmac(KL[4], 1.2190476190476192, Ops::fmac(KL[3], -0.40634920634920635, Ops::fmac(KL[2], 0.4514991181657848, Ops::fmac(KL[1], 0.4514991181657848, Ops::mulc(KL[0], 0.2257495590828924)))))))))))))));
    K[74] = Ops::fmac(KL[16], -0.13544973544973546, Ops::fmac(KL[15], 0.2708994708994709, Ops::fmac(KL[14], 0.045149911816578486, Ops::fmac(KL[10], -0.8126984126984127, Ops::fmac(KL[9], -0.13544973544973546, Ops::fmac(KL[8], -0.4966490299823633, Ops::fmac(KL[7], -0.4514991181657848, Ops::fmac(KL[6], -0.4966490299823633, Ops::fmac(KL[4], -0.40634920634920635, Ops::fmac(KL[3], 0.13544973544973546, Ops::fmac(KL[2], -0.09029982363315697, Ops::fmac(KL[1], -0.09029982363315697, Ops::mulc(KL[0], -0.045149911816578486)))))))))))));
    K[75] = Ops::fmac(KL[17], 0.3160493827160494, Ops::fmac(KL[14], 0.6320987654320988, Ops::fmac(KL[12], 1.2190476190476192, Ops::fmac(KL[11], 0.3160493827160494, Ops::fmac(KL[8], 0.3160493827160494, Ops::fmac(KL[6], 0.40634920634920635, Ops::fmac(KL[5], 3.5668430335097003, Ops::fmac(KL[2], 3.250793650793651, Ops::mulc(KL[0], 2.0317460317460316)))))))));
    K[76] = Ops::fmac(KL[17], 0.045149911816578486, Ops::fmac(KL[14], 0.4740740740740741, Ops::fmac(KL[12], -0.9142857142857143, Ops::fmac(KL[11], -0.18059964726631395, Ops::fmac(KL[8], 0.022574955908289243, Ops::fmac(KL[6], -0.23703703703703705, Ops::fmac(KL[5], -1.3883597883597885, Ops::fmac(KL[2], 0.5530864197530864, Ops::mulc(KL[0], -0.1693121693121693)))))))));
    K[77] = Ops::fmac(KL[14], -0.3160493827160494, Ops::fmac(KL[12], 0.5869488536155203, Ops::fmac(KL[11], 0.09029982363315697, Ops::fmac(KL[8], -0.045149911816578486, Ops::fmac(KL[6], 0.09029982363315697, Ops::fmac(KL[5], 0.5869488536155203, Ops::mulc(KL[2], -0.3160493827160494)))))));
    K[78] = Ops::fmac(KL[17], 0.022574955908289243, Ops::fmac(KL[16], 0.045149911816578486, Ops::fmac(KL[14], 0.045149911816578486, Ops::fmac(KL[13], 0.13544973544973546, Ops::fmac(KL[11], 0.09029982363315697, Ops::fmac(KL[10], 0.06772486772486773, Ops::fmac(KL[8], 0.09029982363315697, Ops::fmac(KL[7], 0.13544973544973546, Ops::fmac(KL[5], 0.09029982363315697, Ops::fmac(KL[4], 0.09029982363315697, Ops::fmac(KL[2], 0.06772486772486773, Ops::mulc(KL[1], 0.13544973544973546))))))))))));
    K[79] = Ops::fmac(KL[17], 0.02821869488536155, Ops::fmac(KL[16], 0.033862433862433865, Ops::fmac(KL[14], 0.10158730158730159, Ops::fmac(KL[13], 0.1693121693121693, Ops::fmac(KL[11], 0.033862433862433865, Ops::fmac(KL[10], 0.02821869488536155, Ops::fmac(KL[8], 0.1693121693121693, Ops::fmac(KL[7], 0.1693121693121693, Ops::fmac(KL[5], 0.022574955908289243, Ops::fmac(KL[4], 0.022574955908289243, Ops::fmac(KL[2], -0.050793650793650794, Ops::mulc(KL[1], -0.033862433862433865))))))))))));
    K[80] = Ops::fmac(KL[17], 0.06772486772486773, Ops::fmac(KL[16], 0.09029982363315697, Ops::fmac(KL[14], 0.40634920634920635, Ops::fmac(KL[13], 0.5869488536155203, Ops::fmac(KL[11], 0.045149911816578486, Ops::fmac(KL[10], 0.022574955908289243, Ops::fmac(KL[8], 0.13544973544973546, Ops::fmac(KL[7], 0.09029982363315697, Ops::fmac(KL[5], 0.09029982363315697, Ops::fmac(KL[4], 0.09029982363315697, Ops::mulc(KL[2], -0.06772486772486773)))))))))));
    K[81] = Ops::fmac(KL[17], 0.2257495590828924, Ops::fmac(KL[16], 0.4514991181657848, Ops::fmac(KL[14], 0.4514991181657848, Ops::fmac(KL[13], 1.2190476190476192, Ops::fmac(KL[12], -0.40634920634920635, Ops::fmac(KL[11], 0.4514991181657848, Ops::fmac(KL[10], 0.2257495590828924, Ops::fmac(KL[8], 0.4514991181657848, Ops::fmac(KL[7], 0.40634920634920635, Ops::fmac(KL[6], -0.2708994708994709, Ops::fmac(KL[5], 2.5735449735449736, Ops::fmac(KL[4], 2.5735449735449736, Ops::fmac(KL[2], 2.347795414462081, Ops::fmac(KL[1], 3.5216931216931218, Ops::mulc(KL[0], 0.9481481481481482)))))))))))))));
    K[82] = Ops::fmac(KL[17], -0.045149911816578486, Ops::fmac(KL[16], -0.09029982363315697, Ops::fmac(KL[14], -0.09029982363315697, Ops::fmac(KL[13], -0.40634920634920635, Ops::fmac(KL[12], 0.13544973544973546, Ops::fmac(KL[10], 0.045149911816578486, Ops::fmac(KL[7], -0.13544973544973546, Ops::fmac(KL[6], 0.2708994708994709, Ops::fmac(KL[5], -0.4966490299823633, Ops::fmac(KL[4], -0.4966490299823633, Ops::fmac(KL[2], -0.4514991181657848, Ops::fmac(KL[1], -0.8126984126984127, Ops::mulc(KL[0], -0.13544973544973546)))))))))))));
    K[83] = Ops::fmac(KL[17], 0.045149911816578486, Ops::fmac(KL[13], -0.40634920634920635, Ops::fmac(KL[12], 0.6772486772486772, Ops::fmac(KL[11], -0.09029982363315697, Ops::fmac(KL[10], -0.045149911816578486, Ops::fmac(KL[8], -0.09029982363315697, Ops::fmac(KL[7], -0.13544973544973546, Ops::fmac(KL[6], 0.2708994708994709, Ops::fmac(KL[5], -0.4966490299823633, Ops::fmac(KL[4], -0.4966490299823633, Ops::fmac(KL[2], 0.09029982363315697, Ops::fmac(KL[1], -0.2708994708994709, Ops::mulc(KL[0], -0.13544973544973546)))))))))))));
    K[84] = Ops::fmac(KL[17], 1.2444444444444445, Ops::fmac(KL[14], 1.7777777777777777, Ops::fmac(KL[12], 3.157671957671958, Ops::fmac(KL[11], 0.49947089947089945, Ops::fmac(KL[8], 0.33015873015873015, Ops::fmac(KL[6], 0.49947089947089945, Ops::fmac(KL[5], 3.157671957671958, Ops::fmac(KL[2], 1.7777777777777777, Ops::mulc(KL[0], 1.2444444444444445)))))))));
    K[85] = Ops::fmac(KL[17], -0.1693121693121693, Ops::fmac(KL[14], 0.5530864197530864, Ops::fmac(KL[12], -1.3883597883597885, Ops::fmac(KL[11], -0.23703703703703705, Ops::fmac(KL[8], 0.022574955908289243, Ops::fmac(KL[6], -0.18059964726631395, Ops::fmac(KL[5], -0.9142857142857143, Ops::fmac(KL[2], 0.4740740740740741, Ops::mulc(KL[0], 0.045149911816578486)))))))));
    K[86] = Ops::fmac(KL[17], 0.02821869488536155, Ops::fmac(KL[16], 0.10158730158730159, Ops::fmac(KL[14], 0.033862433862433865, Ops::fmac(KL[13], 0.1693121693121693, Ops::fmac(KL[11], 0.022574955908289243, Ops::fmac(KL[10], -0.050793650793650794, Ops::fmac(KL[8], 0.022574955908289243, Ops::fmac(KL[7], -0.033862433862433865, Ops::fmac(KL[5], 0.033862433862433865, Ops::fmac(KL[4], 0.1693121693121693, Ops::fmac(KL[2], 0.02821869488536155, Ops::mulc(KL[1], 0.1693121693121693))))))))))));
    K[87] = Ops::fmac(KL[17], -0.10582010582010581, Ops::fmac(KL[16], -0.16084656084656085, Ops::fmac(KL[14], -0.16084656084656085, Ops::fmac(KL[13], -0.364021164021164, Ops::fmac(KL[11], -0.09312169312169312, Ops::fmac(KL[10], -0.10582010582010581, Ops::fmac(KL[8], -0.12698412698412698, Ops::fmac(KL[7], -0.21164021164021163, Ops::fmac(KL[5], -0.09312169312169312, Ops::fmac(KL[4], -0.12698412698412698, Ops::fmac(KL[2], -0.10582010582010581, Ops::mulc(KL[1], -0.21164021164021163))))))))))));
    K[88] = Ops::fmac(KL[17], -0.3216931216931217, Ops::fmac(KL[16], -0.4289241622574956, Ops::fmac(KL[14], -0.7788359788359789, Ops::fmac(KL[13], -1.3883597883597885, Ops::fmac(KL[11], -0.1693121693121693, Ops::fmac(KL[10], -0.062081128747795415, Ops::fmac(KL[8], -0.23703703703703705, Ops::fmac(KL[7], -0.18059964726631395, Ops::fmac(KL[5], -0.23703703703703705, Ops::fmac(KL[4], -0.10158730158730159, Ops::fmac(KL[2], 0.08465608465608465, Ops::mulc(KL[1], 0.045149911816578486))))))))))));
    K[89] = Ops::fmac(KL[17], 0.3724867724867725, Ops::fmac(KL[16], 1.8285714285714285, Ops::fmac(KL[14], 1.0158730158730158, Ops::fmac(KL[13], 1.1174603174603175, Ops::fmac(KL[12], 1.6592592592592592, Ops::fmac(KL[11], -0.3386243386243386, Ops::fmac(KL[10], 0.3724867724867725, Ops::fmac(KL[8], 0.20317460317460317, Ops::fmac(KL[7], 0.10158730158730159, Ops::fmac(KL[6], 0.4740740740740741, Ops::fmac(KL[5], -1.0497354497354496, Ops::fmac(KL[4], 2.471957671957672, Ops::fmac(KL[2], 0.6095238095238096, Ops::fmac(KL[1], 0.6095238095238096, Ops::mulc(KL[0], 0.5079365079365079)))))))))))))));
    K[90] = Ops::fmac(KL[17], -0.1693121693121693, Ops::fmac(KL[16], -0.6095238095238096, Ops::fmac(KL[14], -0.3386243386243386, Ops::fmac(KL[13], -0.7788359788359789, Ops::fmac(KL[12], -0.23703703703703705, Ops::fmac(KL[11], -0.20317460317460317, Ops::fmac(KL[10], -0.033862433862433865, Ops::fmac(KL[8], -0.3386243386243386, Ops::fmac(KL[7], -0.033862433862433865, Ops::fmac(KL[6], -0.20317460317460317, Ops::fmac(KL[5], -0.23703703703703705, Ops::fmac(KL[4], -0.7788359788359789, Ops::fmac(KL[2], -0.3386243386243386, Ops::fmac(KL[1], -0.6095238095238096, Ops::mulc(KL[0], -0.1693121693121693)))))))))))))));
    K[91] = Ops::fmac(KL[17], 0.5079365079365079, Ops::fmac(KL[16], 0.6095238095238096, Ops::fmac(KL[14], 0.6095238095238096, Ops::fmac(KL[13], 2.471957671957672, Ops::fmac(KL[12], -1.0497354497354496, Ops::fmac(KL[11], 0.4740740740740741, Ops::fmac(KL[10], 0.10158730158730159, Ops::fmac(KL[8], 0.20317460317460317, Ops::fmac(KL[7], 0.3724867724867725, Ops::fmac(KL[6], -0.3386243386243386, Ops::fmac(KL[5], 1.6592592592592592, Ops::fmac(KL[4], 1.1174603174603175, Ops::fmac(KL[2], 1.0158730158730158, Ops::fmac(KL[1], 1.8285714285714285, Ops::mulc(KL[0], 0.3724867724867725)))))))))))))));
    K[92] = Ops::fmac(KL[17], 2.0317460317460316, Ops::fmac(KL[14], 3.250793650793651, Ops::fmac(KL[12], 3.5668430335097003, Ops::fmac(KL[11], 0.40634920634920635, Ops::fmac(KL[8], 0.3160493827160494, Ops::fmac(KL[6], 0.3160493827160494, Ops::fmac(KL[5], 1.2190476190476192, Ops::fmac(KL[2], 0.6320987654320988, Ops::mulc(KL[0], 0.3160493827160494)))))))));
    K[93] = Ops::fmac(KL[17], 0.06772486772486773, Ops::fmac(KL[16], 0.40634920634920635, Ops::fmac(KL[14], 0.09029982363315697, Ops::fmac(KL[13], 0.5869488536155203, Ops::fmac(KL[11], 0.09029982363315697, Ops::fmac(KL[10], -0.06772486772486773, Ops::fmac(KL[8], 0.09029982363315697, Ops::fmac(KL[5], 0.045149911816578486, Ops::fmac(KL[4], 0.13544973544973546, Ops::fmac(KL[2], 0.022574955908289243, Ops::mulc(KL[1], 0.09029982363315697)))))))))));
    K[94] = Ops::fmac(KL[17], -0.3216931216931217, Ops::fmac(KL[16], -0.7788359788359789, Ops::fmac(KL[14], -0.4289241622574956, Ops::fmac(KL[13], -1.3883597883597885, Ops::fmac(KL[11], -0.23703703703703705, Ops::fmac(KL[10], 0.08465608465608465, Ops::fmac(KL[8], -0.10158730158730159, Ops::fmac(KL[7], 0.045149911816578486, Ops::fmac(KL[5], -0.1693121693121693, Ops::fmac(KL[4], -0.23703703703703705, Ops::fmac(KL[2], -0.062081128747795415, Ops::mulc(KL[1], -0.18059964726631395))))))))))));
    K[95] = Ops::fmac(KL[17], 1.0158730158730158, Ops::fmac(KL[16], 1.6253968253968254, Ops::fmac(KL[14], 1.6253968253968254, Ops::fmac(KL[13], 3.5668430335097003, Ops::fmac(KL[11], 0.40634920634920635, Ops::fmac(KL[10], 0.1580246913580247, Ops::fmac(KL[8], 0.3160493827160494, Ops::fmac(KL[7], 0.3160493827160494, Ops::fmac(KL[5], 0.40634920634920635, Ops::fmac(KL[4], 0.3160493827160494, Ops::fmac(KL[2], 0.1580246913580247, Ops::mulc(KL[1], 0.3160493827160494))))))))))));
    K[96] = Ops::fmac(KL[17], -0.13544973544973546, Ops::fmac(KL[16], -0.2708994708994709, Ops::fmac(KL[14], 0.09029982363315697, Ops::fmac(KL[13], -0.4966490299823633, Ops::fmac(KL[12], -0.4966490299823633, Ops::fmac(KL[11], 0.2708994708994709, Ops::fmac(KL[10], -0.13544973544973546, Ops::fmac(KL[8], -0.09029982363315697, Ops::fmac(KL[7], -0.045149911816578486, Ops::fmac(KL[6], -0.09029982363315697, Ops::fmac(KL[5], 0.6772486772486772, Ops::fmac(KL[4], -0.40634920634920635, Ops::mulc(KL[0], 0.045149911816578486)))))))))))));
    K[97] = Ops::fmac(KL[17], -0.13544973544973546, Ops::fmac(KL[16], -0.8126984126984127, Ops::fmac(KL[14], -0.4514991181657848, Ops::fmac(KL[13], -0.4966490299823633, Ops::fmac(KL[12], -0.4966490299823633, Ops::fmac(KL[11], 0.2708994708994709, Ops::fmac(KL[10], -0.13544973544973546, Ops::fmac(KL[7], 0.045149911816578486, Ops::fmac(KL[5], 0.13544973544973546, Ops::fmac(KL[4], -0.40634920634920635, Ops::fmac(KL[2], -0.09029982363315697, Ops::fmac(KL[1], -0.09029982363315697, Ops::mulc(KL[0], -0.045149911816578486)))))))))))));
    K[98] = Ops::fmac(KL[17], 0.9481481481481482, Ops::fmac(KL[16], 3.5216931216931218, Ops::fmac(KL[14], 2.347795414462081, Ops::fmac(KL[13], 2.5735449735449736, Ops::fmac(KL[12], 2.5735449735449736, Ops::fmac(KL[11], -0.2708994708994709, Ops::fmac(KL[10], 0.40634920634920635, Ops::fmac(KL[8], 0.4514991181657848, Ops::fmac(KL[7], 0.2257495590828924, Ops::fmac(KL[6], 0.4514991181657848, Ops::fmac(KL[5], -0.40634920634920635, Ops::fmac(KL[4], 1.2190476190476192, Ops::fmac(KL[2], 0.4514991181657848, Ops::fmac(KL[1], 0.4514991181657848, Ops::mulc(KL[0], 0.2257495590828924)))))))))))))));
    K[99] = Ops::fmac(KL[17], 0.3160493827160494, Ops::fmac(KL[16], 0.6320987654320988, Ops::fmac(KL[15], 1.2190476190476192, Ops::fmac(KL[11], 3.5668430335097003, Ops::fmac(KL[10], 3.250793650793651, Ops::fmac(KL[9], 2.0317460317460316, Ops::fmac(KL[5], 0.3160493827160494, Ops::fmac(KL[4], 0.3160493827160494, Ops::mulc(KL[3], 0.40634920634920635)))))))));
    K[100] = Ops::fmac(KL[17], 0.045149911816578486, Ops::fmac(KL[16], 0.4740740740740741, Ops::fmac(KL[15], -0.9142857142857143, Ops::fmac(KL[11], -1.3883597883597885, Ops::fmac(KL[10], 0.5530864197530864, Ops::fmac(KL[9], -0.1693121693121693, Ops::fmac(KL[5], -0.18059964726631395, Ops::fmac(KL[4], 0.022574955908289243, Ops::mulc(KL[3], -0.23703703703703705)))))))));
    K[101] = Ops::fmac(KL[16], -0.3160493827160494, Ops::fmac(KL[15], 0.5869488536155203, Ops::fmac(KL[11], 0.5869488536155203, Ops::fmac(KL[10], -0.3160493827160494, Ops::fmac(KL[5], 0.09029982363315697, Ops::fmac(KL[4], -0.045149911816578486, Ops::mulc(KL[3], 0.09029982363315697)))))));
    K[102] = Ops::fmac(KL[17], -0.045149911816578486, Ops::fmac(KL[16], -0.09029982363315697, Ops::fmac(KL[15], 0.13544973544973546, Ops::fmac(KL[14], -0.09029982363315697, Ops::fmac(KL[13], -0.40634920634920635, Ops::fmac(KL[11], -0.4966490299823633, Ops::fmac(KL[10], -0.4514991181657848, Ops::fmac(KL[9], -0.13544973544973546, Ops::fmac(KL[8], -0.4966490299823633, Ops::fmac(KL[7], -0.8126984126984127, Ops::fmac(KL[3], 0.2708994708994709, Ops::fmac(KL[2], 0.045149911816578486, Ops::mulc(KL[1], -0.13544973544973546)))))))))))));
    K[103] = Ops::fmac(KL[17], 0.2257495590828924, Ops::fmac(KL[16], 0.4514991181657848, Ops::fmac(KL[15], -0.40634920634920635, Ops::fmac(KL[14], 0.4514991181657848, Ops::fmac(KL[13], 1.2190476190476192, Ops::fmac(KL[11], 2.5735449735449736, Ops::fmac(KL[10], 2.347795414462081, Ops::fmac(KL[9], 0.9481481481481482, Ops::fmac(KL[8], 2.5735449735449736, Ops::fmac(KL[7], 3.5216931216931218, Ops::fmac(KL[5], 0.4514991181657848, Ops::fmac(KL[4], 0.4514991181657848, Ops::fmac(KL[3], -0.2708994708994709, Ops::fmac(KL[2], 0.2257495590828924, Ops::mulc(KL[1], 0.40634920634920635)))))))))))))));
    K[104] = Ops::fmac(KL[17], 0.045149911816578486, Ops::fmac(KL[15], 0.6772486772486772, Ops::fmac(KL[13], -0.40634920634920635, Ops::fmac(KL[11], -0.4966490299823633, Ops::fmac(KL[10], 0.09029982363315697, Ops::fmac(KL[9], -0.13544973544973546, Ops::fmac(KL[8], -0.4966490299823633, Ops::fmac(KL[7], -0.2708994708994709, Ops::fmac(KL[5], -0.09029982363315697, Ops::fmac(KL[4], -0.09029982363315697, Ops::fmac(KL[3], 0.2708994708994709, Ops::fmac(KL[2], -0.045149911816578486, Ops::mulc(KL[1], -0.13544973544973546)))))))))))));
    K[105] = Ops::fmac(KL[17], 1.2444444444444445, Ops::fmac(KL[16], 1.7777777777777777, Ops::fmac(KL[15], 3.157671957671958, Ops::fmac(KL[11], 3.157671957671958, Ops::fmac(KL[10], 1.7777777777777777, Ops::fmac(KL[9], 1.2444444444444445, Ops::fmac(KL[5], 0.49947089947089945, Ops::fmac(KL[4], 0.33015873015873015, Ops::mulc(KL[3], 0.49947089947089945)))))))));
    K[106] = Ops::fmac(KL[17], -0.1693121693121693, Ops::fmac(KL[16], 0.5530864197530864, Ops::fmac(KL[15], -1.3883597883597885, Ops::fmac(KL[11], -0.9142857142857143, Ops::fmac(KL[10], 0.4740740740740741, Ops::fmac(KL[9], 0.045149911816578486, Ops::fmac(KL[5], -0.23703703703703705, Ops::fmac(KL[4], 0.022574955908289243, Ops::mulc(KL[3], -0.18059964726631395)))))))));
    K[107] = Ops::fmac(KL[17], -0.1693121693121693, Ops::fmac(KL[16], -0.3386243386243386, Ops::fmac(KL[15], -0.23703703703703705, Ops::fmac(KL[14], -0.6095238095238096, Ops::fmac(KL[13], -0.7788359788359789, Ops::fmac(KL[11], -0.23703703703703705, Ops::fmac(KL[10], -0.3386243386243386, Ops::fmac(KL[9], -0.1693121693121693, Ops::fmac(KL[8], -0.7788359788359789, Ops::fmac(KL[7], -0.6095238095238096, Ops::fmac(KL[5], -0.20317460317460317, Ops::fmac(KL[4], -0.3386243386243386, Ops::fmac(KL[3], -0.20317460317460317, Ops::fmac(KL[2], -0.033862433862433865, Ops::mulc(KL[1], -0.033862433862433865)))))))))))))));
    K[108] = Ops::fmac(KL[17], 0.3724867724867725, Ops::fmac(KL[16], 1.0158730158730158, Ops::fmac(KL[15], 1.6592592592592592, Ops::fmac(KL[14], 1.8285714285714285, Ops::fmac(KL[13], 1.1174603174603175, Ops::fmac(KL[11], -1.0497354497354496, Ops::fmac(KL[10], 0.6095238095238096, Ops::fmac(KL[9], 0.5079365079365079, Ops::fmac(KL[8], 2.471957671957672, Ops::fmac(KL[7], 0.6095238095238096, Ops::fmac(KL[5], -0.3386243386243386, Ops::fmac(KL[4], 0.20317460317460317, Ops::fmac(KL[3], 0.4740740740740741, Ops::fmac(KL[2], 0.3724867724867725, Ops::mulc(KL[1], 0.10158730158730159)))))))))))))));
    K[109] = Ops::fmac(KL[17], 0.5079365079365079, Ops::fmac(KL[16], 0.6095238095238096, Ops::fmac(KL[15], -1.0497354497354496, Ops::fmac(KL[14], 0.6095238095238096, Ops::fmac(KL[13], 2.471957671957672, Ops::fmac(KL[11], 1.6592592592592592, Ops::fmac(KL[10], 1.0158730158730158, Ops::fmac(KL[9], 0.3724867724867725, Ops::fmac(KL[8], 1.1174603174603175, Ops::fmac(KL[7], 1.8285714285714285, Ops::fmac(KL[5], 0.4740740740740741, Ops::fmac(KL[4], 0.20317460317460317, Ops::fmac(KL[3], -0.3386243386243386, Ops::fmac(KL[2], 0.10158730158730159, Ops::mulc(KL[1], 0.3724867724867725)))))))))))))));
    K[110] = Ops::fmac(KL[17], 2.0317460317460316, Ops::fmac(KL[16], 3.250793650793651, Ops::fmac(KL[15], 3.5668430335097003, Ops::fmac(KL[11], 1.2190476190476192, Ops::fmac(KL[10], 0.6320987654320988, Ops::fmac(KL[9], 0.3160493827160494, Ops::fmac(KL[5], 0.40634920634920635, Ops::fmac(KL[4], 0.3160493827160494, Ops::mulc(KL[3], 0.3160493827160494)))))))));
    K[111] = Ops::fmac(KL[17], -0.13544973544973546, Ops::fmac(KL[16], -0.4514991181657848, Ops::fmac(KL[15], -0.4966490299823633, Ops::fmac(KL[14], -0.8126984126984127, Ops::fmac(KL[13], -0.4966490299823633, Ops::fmac(KL[11], 0.13544973544973546, Ops::fmac(KL[10], -0.09029982363315697, Ops::fmac(KL[9], -0.045149911816578486, Ops::fmac(KL[8], -0.40634920634920635, Ops::fmac(KL[7], -0.09029982363315697, Ops::fmac(KL[5], 0.2708994708994709, Ops::fmac(KL[2], -0.13544973544973546, Ops::mulc(KL[1], 0.045149911816578486)))))))))))));
    K[112] = Ops::fmac(KL[17], -0.13544973544973546, Ops::fmac(KL[16], 0.09029982363315697, Ops::fmac(KL[15], -0.4966490299823633, Ops::fmac(KL[14], -0.2708994708994709, Ops::fmac(KL[13], -0.4966490299823633, Ops::fmac(KL[11], 0.6772486772486772, Ops::fmac(KL[9], 0.045149911816578486, Ops::fmac(KL[8], -0.40634920634920635, Ops::fmac(KL[5], 0.2708994708994709, Ops::fmac(KL[4], -0.09029982363315697, Ops::fmac(KL[3], -0.09029982363315697, Ops::fmac(KL[2], -0.13544973544973546, Ops::mulc(KL[1], -0.045149911816578486)))))))))))));
    K[113] = Ops::fmac(KL[17], 0.9481481481481482, Ops::fmac(KL[16], 2.347795414462081, Ops::fmac(KL[15], 2.5735449735449736, Ops::fmac(KL[14], 3.5216931216931218, Ops::fmac(KL[13], 2.5735449735449736, Ops::fmac(KL[11], -0.40634920634920635, Ops::fmac(KL[10], 0.4514991181657848, Ops::fmac(KL[9], 0.2257495590828924, Ops::fmac(KL[8], 1.2190476190476192, Ops::fmac(KL[7], 0.4514991181657848, Ops::fmac(KL[5], -0.2708994708994709, Ops::fmac(KL[4], 0.4514991181657848, Ops::fmac(KL[3], 0.4514991181657848, Ops::fmac(KL[2], 0.40634920634920635, Ops::mulc(KL[1], 0.2257495590828924)))))))))))))));
    K[114] = Ops::fmac(KL[17], 1.0835978835978837, Ops::fmac(KL[16], 2.1671957671957673, Ops::fmac(KL[15], 3.250793650793651, Ops::fmac(KL[14], 2.1671957671957673, Ops::fmac(KL[13], 3.250793650793651, Ops::fmac(KL[12], 3.7925925925925927, Ops::fmac(KL[11], 3.250793650793651, Ops::fmac(KL[10], 2.1671957671957673, Ops::fmac(KL[9], 1.0835978835978837, Ops::fmac(KL[8], 3.250793650793651, Ops::fmac(KL[7], 2.1671957671957673, Ops::fmac(KL[6], 3.7925925925925927, Ops::fmac(KL[5], 7.0433862433862435, Ops::fmac(KL[4], 7.0433862433862435, Ops::fmac(KL[3], 7.0433862433862435, Ops::fmac(KL[2], 5.95978835978836, Ops::fmac(KL[1], 5.95978835978836, Ops::mulc(KL[0], 3.7925925925925927))))))))))))))))));
    K[115] = Ops::fmac(KL[15], -0.8126984126984127, Ops::fmac(KL[13], 1.0835978835978837, Ops::fmac(KL[12], -0.8126984126984127, Ops::fmac(KL[11], 0.8126984126984127, Ops::fmac(KL[10], 0.8126984126984127, Ops::fmac(KL[9], 0.2708994708994709, Ops::fmac(KL[8], 0.8126984126984127, Ops::fmac(KL[7], 1.8962962962962964, Ops::fmac(KL[6], -1.0835978835978837, Ops::fmac(KL[5], 0.8126984126984127, Ops::fmac(KL[4], 0.8126984126984127, Ops::fmac(KL[3], -1.0835978835978837, Ops::fmac(KL[2], 0.8126984126984127, Ops::fmac(KL[1], 1.8962962962962964, Ops::mulc(KL[0], 0.2708994708994709)))))))))))))));
    K[116] = Ops::fmac(KL[17], 0.2708994708994709, Ops::fmac(KL[16], 0.8126984126984127, Ops::fmac(KL[15], 0.8126984126984127, Ops::fmac(KL[14], 1.8962962962962964, Ops::fmac(KL[13], 0.8126984126984127, Ops::fmac(KL[12], -1.0835978835978837, Ops::fmac(KL[11], -0.8126984126984127, Ops::fmac(KL[8], 1.0835978835978837, Ops::fmac(KL[6], -0.8126984126984127, Ops::fmac(KL[5], -1.0835978835978837, Ops::fmac(KL[4], 0.8126984126984127, Ops::fmac(KL[3], 0.8126984126984127, Ops::fmac(KL[2], 1.8962962962962964, Ops::fmac(KL[1], 0.8126984126984127, Ops::mulc(KL[0], 0.2708994708994709)))))))))))))));
    K[117] = Ops::fmac(KL[17], 1.0835978835978837, Ops::fmac(KL[16], 2.1671957671957673, Ops::fmac(KL[15], 3.7925925925925927, Ops::fmac(KL[14], 2.1671957671957673, Ops::fmac(KL[13], 3.250793650793651, Ops::fmac(KL[12], 3.250793650793651, Ops::fmac(KL[11], 7.0433862433862435, Ops::fmac(KL[10], 5.95978835978836, Ops::fmac(KL[9], 3.7925925925925927, Ops::fmac(KL[8], 7.0433862433862435, Ops::fmac(KL[7], 5.95978835978836, Ops::fmac(KL[6], 7.0433862433862435, Ops::fmac(KL[5], 3.250793650793651, Ops::fmac(KL[4], 3.250793650793651, Ops::fmac(KL[3], 3.7925925925925927, Ops::fmac(KL[2], 2.1671957671957673, Ops::fmac(KL[1], 2.1671957671957673, Ops::mulc(KL[0], 1.0835978835978837))))))))))))))))));
    K[118] = Ops::fmac(KL[17], 0.2708994708994709, Ops::fmac(KL[16], 1.8962962962962964, Ops::fmac(KL[15], -1.0835978835978837, Ops::fmac(KL[14], 0.8126984126984127, Ops::fmac(KL[13], 0.8126984126984127, Ops::fmac(KL[12], 0.8126984126984127, Ops::fmac(KL[11], -1.0835978835978837, Ops::fmac(KL[10], 1.8962962962962964, Ops::fmac(KL[9], 0.2708994708994709, Ops::fmac(KL[8], 0.8126984126984127, Ops::fmac(KL[7], 0.8126984126984127, Ops::fmac(KL[6], 0.8126984126984127, Ops::fmac(KL[5], -0.8126984126984127, Ops::fmac(KL[4], 1.0835978835978837, Ops::mulc(KL[3], -0.8126984126984127)))))))))))))));
    K[119] = Ops::fmac(KL[17], 3.7925925925925927, Ops::fmac(KL[16], 5.95978835978836, Ops::fmac(KL[15], 7.0433862433862435, Ops::fmac(KL[14], 5.95978835978836, Ops::fmac(KL[13], 7.0433862433862435, Ops::fmac(KL[12], 7.0433862433862435, Ops::fmac(KL[11], 3.7925925925925927, Ops::fmac(KL[10], 2.1671957671957673, Ops::fmac(KL[9], 1.0835978835978837, Ops::fmac(KL[8], 3.250793650793651, Ops::fmac(KL[7], 2.1671957671957673, Ops::fmac(KL[6], 3.250793650793651, Ops::fmac(KL[5], 3.7925925925925927, Ops::fmac(KL[4], 3.250793650793651, Ops::fmac(KL[3], 3.250793650793651, Ops::fmac(KL[2], 2.1671957671957673, Ops::fmac(KL[1], 2.1671957671957673, Ops::mulc(KL[0], 1.0835978835978837))))))))))))))))));
  }
  static constexpr int TERMS = 1215;
};

template <> struct Kappa<3, 1> {
  static constexpr int NKL = 40;
  // K[u] = sum_{k,(m<=n)} KL[k*NLAM + mn] * C[k][mn][i][j], KL = kappa_k * Lam_mn
  template <class Ops> __device__ __forceinline__ static void upper(const typename Ops::T* KL, typename Ops::T* K) {
    K[0] = Ops::fmac(KL[30], 0.25, Ops::fmac(KL[20], 0.25, Ops::fmac(KL[10], 0.25, Ops::mulc(KL[0], 0.25))));
    K[1] = Ops::fmac(KL[31], 0.25, Ops::fmac(KL[21], 0.25, Ops::fmac(KL[11], 0.25, Ops::mulc(KL[1], 0.25))));
    K[2] = Ops::fmac(KL[32], 0.25, Ops::fmac(KL[22], 0.25, Ops::fmac(KL[12], 0.25, Ops::mulc(KL[2], 0.25))));
    K[3] = Ops::fmac(KL[33], 0.25, Ops::fmac(KL[23], 0.25, Ops::fmac(KL[13], 0.25, Ops::mulc(KL[3], 0.25))));
    K[4] = Ops::fmac(KL[34], 0.25, Ops::fmac(KL[24], 0.25, Ops::fmac(KL[14], 0.25, Ops::mulc(KL[4], 0.25))));
    K[5] = Ops::fmac(KL[35], 0.25, Ops::fmac(KL[25], 0.25, Ops::fmac(KL[15], 0.25, Ops::mulc(KL[5], 0.25))));
    K[6] = Ops::fmac(KL[36], 0.25, Ops::fmac(KL[26], 0.25, Ops::fmac(KL[16], 0.25, Ops::mulc(KL[6], 0.25))));
    K[7] = Ops::fmac(KL[37], 0.25, Ops::fmac(KL[27], 0.25, Ops::fmac(KL[17], 0.25, Ops::mulc(KL[7], 0.25))));
    K[8] = Ops::fmac(KL[38], 0.25, Ops::fmac(KL[28], 0.25, Ops::fmac(KL[18], 0.25, Ops::mulc(KL[8], 0.25))));
    K[9] = Ops::fmac(KL[39], 0.25, Ops::fmac(KL[29], 0.25, Ops::fmac(KL[19], 0.25, Ops::mulc(KL[9], 0.25))));
  }
  static constexpr int TERMS = 40;
};

template <> struct Kappa<3, 2> {
  static constexpr int NKL = 40;
  // K[u] = sum_{k,(m<=n)} KL[k*NLAM + mn] * C[k][mn][i][j], KL = kappa_k * Lam_mn
  template <class Ops> __device__ __forceinline__ static void upper(const typename Ops::T* KL, typename Ops::T* K) {
    K[0] = Ops::fmac(KL[30], 0.11666666666666667, Ops::fmac(KL[20], 0.11666666666666667, Ops::fmac(KL[10], 0.11666666666666667, Ops::mulc(KL[0], 0.25))));
    K[1] = Ops::fmac(KL[31], -0.016666666666666666, Ops::fmac(KL[21], -0.016666666666666666, Ops::fmac(KL[11], -0.08333333333333333, Ops::mulc(KL[1], -0.08333333333333333))));
    K[2] = Ops::fmac(KL[32], -0.016666666666666666, Ops::fmac(KL[22], -0.08333333333333333, Ops::fmac(KL[12], -0.016666666666666666, Ops::mulc(KL[2], -0.08333333333333333))));
    K[3] = Ops::fmac(KL[33], -0.08333333333333333, Ops::fmac(KL[23], -0.016666666666666666, Ops::fmac(KL[13], -0.016666666666666666, Ops::mulc(KL[3], -0.08333333333333333))));
    K[4] = Ops::fmac(KL[31], 0.06666666666666667, Ops::fmac(KL[30], -0.06666666666666667, Ops::fmac(KL[21], 0.06666666666666667, Ops::fmac(KL[20], -0.06666666666666667, Ops::fmac(KL[11], 0.06666666666666667, Ops::fmac(KL[10], -0.13333333333333333, Ops::fmac(KL[1], 0.4, Ops::mulc(KL[0], 0.06666666666666667))))))));
    K[5] = Ops::fmac(KL[32], 0.06666666666666667, Ops::fmac(KL[30], -0.06666666666666667, Ops::fmac(KL[22], 0.06666666666666667, Ops::fmac(KL[20], -0.13333333333333333, Ops::fmac(KL[12], 0.06666666666666667, Ops::fmac(KL[10], -0.06666666666666667, Ops::fmac(KL[2], 0.4, Ops::mulc(KL[0], 0.06666666666666667))))))));
    K[6] = Ops::fmac(KL[33], 0.06666666666666667, Ops::fmac(KL[30], -0.13333333333333333, Ops::fmac(KL[23], 0.06666666666666667, Ops::fmac(KL[20], -0.06666666666666667, Ops::fmac(KL[13], 0.06666666666666667, Ops::fmac(KL[10], -0.06666666666666667, Ops::fmac(KL[3], 0.4, Ops::mulc(KL[0], 0.06666666666666667))))))));
    K[7] = Ops::fmac(KL[32], -0.06666666666666667, Ops::fmac(KL[31], -0.06666666666666667, Ops::fmac(KL[22], -0.06666666666666667, Ops::fmac(KL[21], -0.13333333333333333, Ops::fmac(KL[12], -0.13333333333333333, Ops::fmac(KL[11], -0.06666666666666667, Ops::fmac(KL[2], 0.06666666666666667, Ops::mulc(KL[1], 0.06666666666666667))))))));
    K[8] = Ops::fmac(KL[33], -0.06666666666666667, Ops::fmac(KL[31], -0.13333333333333333, Ops::fmac(KL[23], -0.06666666666666667, Ops::fmac(KL[21], -0.06666666666666667, Ops::fmac(KL[13], -0.13333333333333333, Ops::fmac(KL[11], -0.06666666666666667, Ops::fmac(KL[3], 0.06666666666666667, Ops::mulc(KL[1], 0.06666666666666667))))))));
    K[9] = Ops::fmac(KL[33], -0.06666666666666667, Ops::fmac(KL[32], -0.13333333333333333, Ops::fmac(KL[23], -0.13333333333333333, Ops::fmac(KL[22], -0.06666666666666667, Ops::fmac(KL[13], -0.06666666666666667, Ops::fmac(KL[12], -0.06666666666666667, Ops::fmac(KL[3], 0.06666666666666667, Ops::mulc(KL[2], 0.06666666666666667))))))));
    K[10] = Ops::fmac(KL[34], 0.11666666666666667, Ops::fmac(KL[24], 0.11666666666666667, Ops::fmac(KL[14], 0.25, Ops::mulc(KL[4], 0.11666666666666667))));
    K[11] = Ops::fmac(KL[35], -0.016666666666666666, Ops::fmac(KL[25], -0.08333333333333333, Ops::fmac(KL[15], -0.08333333333333333, Ops::mulc(KL[5], -0.016666666666666666))));
    K[12] = Ops::fmac(KL[36], -0.08333333333333333, Ops::fmac(KL[26], -0.016666666666666666, Ops::fmac(KL[16], -0.08333333333333333, Ops::mulc(KL[6], -0.016666666666666666))));
    K[13] = Ops::fmac(KL[34], -0.06666666666666667, Ops::fmac(KL[31], 0.06666666666666667, Ops::fmac(KL[24], -0.06666666666666667, Ops::fmac(KL[21], 0.06666666666666667, Ops::fmac(KL[14], 0.06666666666666667, Ops::fmac(KL[11], 0.4, Ops::fmac(KL[4], -0.13333333333333333, Ops::mulc(KL[1], 0.06666666666666667))))))));
    K[14] = Ops::fmac(KL[35], -0.06666666666666667, Ops::fmac(KL[31], -0.06666666666666667, Ops::fmac(KL[25], -0.06666666666666667, Ops::fmac(KL[21], -0.13333333333333333, Ops::fmac(KL[15], 0.06666666666666667, Ops::fmac(KL[11], 0.06666666666666667, Ops::fmac(KL[5], -0.13333333333333333, Ops::mulc(KL[1], -0.06666666666666667))))))));
    K[15] = Ops::fmac(KL[36], -0.06666666666666667, Ops::fmac(KL[31], -0.13333333333333333, Ops::fmac(KL[26], -0.06666666666666667, Ops::fmac(KL[21], -0.06666666666666667, Ops::fmac(KL[16], 0.06666666666666667, Ops::fmac(KL[11], 0.06666666666666667, Ops::fmac(KL[6], -0.13333333333333333, Ops::mulc(KL[1], -0.06666666666666667))))))));
    K[16] = Ops::fmac(KL[35], 0.06666666666666667, Ops::fmac(KL[34], -0.06666666666666667, Ops::fmac(KL[25], 0.06666666666666667, Ops::fmac(KL[24], -0.13333333333333333, Ops::fmac(KL[15], 0.4, Ops::fmac(KL[14], 0.06666666666666667, Ops::fmac(KL[5], 0.06666666666666667, Ops::mulc(KL[4], -0.06666666666666667))))))));
    K[17] = Ops::fmac(KL[36], 0.06666666666666667, Ops::fmac(KL[34], -0.13333333333333333, Ops::fmac(KL[26], 0.06666666666666667, Ops::fmac(KL[24], -0.06666666666666667, Ops::fmac(KL[16], 0.4, Ops::fmac(KL[14], 0.06666666666666667, Ops::fmac(KL[6], 0.06666666666666667, Ops::mulc(KL[4], -0.06666666666666667))))))));
    K[18] = Ops::fmac(KL[36], -0.06666666666666667, Ops::fmac(KL[35], -0.13333333333333333, Ops::fmac(KL[26], -0.13333333333333333, Ops::fmac(KL[25], -0.06666666666666667, Ops::fmac(KL[16], 0.06666666666666667, Ops::fmac(KL[15], 0.06666666666666667, Ops::fmac(KL[6], -0.06666666666666667, Ops::mulc(KL[5], -0.06666666666666667))))))));
    K[19] = Ops::fmac(KL[37], 0.11666666666666667, Ops::fmac(KL[27], 0.25, Ops::fmac(KL[17], 0.11666666666666667, Ops::mulc(KL[7], 0.11666666666666667))));
    K[20] = Ops::fmac(KL[38], -0.08333333333333333, Ops::fmac(KL[28], -0.08333333333333333, Ops::fmac(KL[18], -0.016666666666666666, Ops::mulc(KL[8], -0.016666666666666666))));
    K[21] = Ops::fmac(KL[35], -0.06666666666666667, Ops::fmac(KL[32], -0.06666666666666667, Ops::fmac(KL[25], 0.06666666666666667, Ops::fmac(KL[22], 0.06666666666666667, Ops::fmac(KL[15], -0.06666666666666667, Ops::fmac(KL[12], -0.13333333333333333, Ops::fmac(KL[5], -0.13333333333333333, Ops::mulc(KL[2], -0.06666666666666667))))))));
    K[22] = Ops::fmac(KL[37], -0.06666666666666667, Ops::fmac(KL[32], 0.06666666666666667, Ops::fmac(KL[27], 0.06666666666666667, Ops::fmac(KL[22], 0.4, Ops::fmac(KL[17], -0.06666666666666667, Ops::fmac(KL[12], 0.06666666666666667, Ops::fmac(KL[7], -0.13333333333333333, Ops::mulc(KL[2], 0.06666666666666667))))))));
    K[23] = Ops::fmac(KL[38], -0.06666666666666667, Ops::fmac(KL[32], -0.13333333333333333, Ops::fmac(KL[28], 0.06666666666666667, Ops::fmac(KL[22], 0.06666666666666667, Ops::fmac(KL[18], -0.06666666666666667, Ops::fmac(KL[12], -0.06666666666666667, Ops::fmac(KL[8], -0.13333333333333333, Ops::mulc(KL[2], -0.06666666666666667))))))));
    K[24] = Ops::fmac(KL[37], -0.06666666666666667, Ops::fmac(KL[35], 0.06666666666666667, Ops::fmac(KL[27], 0.06666666666666667, Ops::fmac(KL[25], 0.4, Ops::fmac(KL[17], -0.13333333333333333, Ops::fmac(KL[15], 0.06666666666666667, Ops::fmac(KL[7], -0.06666666666666667, Ops::mulc(KL[5], 0.06666666666666667))))))));
    K[25] = Ops::fmac(KL[38], -0.06666666666666667, Ops::fmac(KL[35], -0.13333333333333333, Ops::fmac(KL[28], 0.06666666666666667, Ops::fmac(KL[25], 0.06666666666666667, Ops::fmac(KL[18], -0.13333333333333333, Ops::fmac(KL[15], -0.06666666666666667, Ops::fmac(KL[8], -0.06666666666666667, Ops::mulc(KL[5], -0.06666666666666667))))))));
    K[26] = Ops::fmac(KL[38], 0.06666666666666667, Ops::fmac(KL[37], -0.13333333333333333, Ops::fmac(KL[28], 0.4, Ops::fmac(KL[27], 0.06666666666666667, Ops::fmac(KL[18], 0.06666666666666667, Ops::fmac(KL[17], -0.06666666666666667, Ops::fmac(KL[8], 0.06666666666666667, Ops::mulc(KL[7], -0.06666666666666667))))))));
    K[27] = Ops::fmac(KL[39], 0.25, Ops::fmac(KL[29], 0.11666666666666667, Ops::fmac(KL[19], 0.11666666666666667, Ops::mulc(KL[9], 0.11666666666666667))));
    K[28] = Ops::fmac(KL[36], 0.06666666666666667, Ops::fmac(KL[33], 0.06666666666666667, Ops::fmac(KL[26], -0.06666666666666667, Ops::fmac(KL[23], -0.06666666666666667, Ops::fmac(KL[16], -0.06666666666666667, Ops::fmac(KL[13], -0.13333333333333333, Ops::fmac(KL[6], -0.13333333333333333, Ops::mulc(KL[3], -0.06666666666666667))))))));
    K[29] = Ops::fmac(KL[38], 0.06666666666666667, Ops::fmac(KL[33], 0.06666666666666667, Ops::fmac(KL[28], -0.06666666666666667, Ops::fmac(KL[23], -0.13333333333333333, Ops::fmac(KL[18], -0.06666666666666667, Ops::fmac(KL[13], -0.06666666666666667, Ops::fmac(KL[8], -0.13333333333333333, Ops::mulc(KL[3], -0.06666666666666667))))))));
    K[30] = Ops::fmac(KL[39], 0.06666666666666667, Ops::fmac(KL[33], 0.4, Ops::fmac(KL[29], -0.06666666666666667, Ops::fmac(KL[23], 0.06666666666666667, Ops::fmac(KL[19], -0.06666666666666667, Ops::fmac(KL[13], 0.06666666666666667, Ops::fmac(KL[9], -0.13333333333333333, Ops::mulc(KL[3], 0.06666666666666667))))))));
    K[31] = Ops::fmac(KL[38], 0.06666666666666667, Ops::fmac(KL[36], 0.06666666666666667, Ops::fmac(KL[28], -0.06666666666666667, Ops::fmac(KL[26], -0.13333333333333333, Ops::fmac(KL[18], -0.13333333333333333, Ops::fmac(KL[16], -0.06666666666666667, Ops::fmac(KL[8], -0.06666666666666667, Ops::mulc(KL[6], -0.06666666666666667))))))));
    K[32] = Ops::fmac(KL[39], 0.06666666666666667, Ops::fmac(KL[36], 0.4, Ops::fmac(KL[29], -0.06666666666666667, Ops::fmac(KL[26], 0.06666666666666667, Ops::fmac(KL[19], -0.13333333333333333, Ops::fmac(KL[16], 0.06666666666666667, Ops::fmac(KL[9], -0.06666666666666667, Ops::mulc(KL[6], 0.06666666666666667))))))));
    K[33] = Ops::fmac(KL[39], 0.06666666666666667, Ops::fmac(KL[38], 0.4, Ops::fmac(KL[29], -0.13333333333333333, Ops::fmac(KL[28], 0.06666666666666667, Ops::fmac(KL[19], -0.06666666666666667, Ops::fmac(KL[18], 0.06666666666666667, Ops::fmac(KL[9], -0.06666666666666667, Ops::mulc(KL[8], 0.06666666666666667))))))));
    K[34] = Ops::fmac(KL[34], 0.26666666666666666, Ops::fmac(KL[31], 0.26666666666666666, Ops::fmac(KL[30], 0.26666666666666666, Ops::fmac(KL[24], 0.26666666666666666, Ops::fmac(KL[21], 0.26666666666666666, Ops::fmac(KL[20], 0.26666666666666666, Ops::fmac(KL[14], 0.26666666666666666, Ops::fmac(KL[11], 0.5333333333333333, Ops::fmac(KL[10], 0.8, Ops::fmac(KL[4], 0.8, Ops::fmac(KL[1], 0.5333333333333333, Ops::mulc(KL[0], 0.26666666666666666))))))))))));
    K[35] = Ops::fmac(KL[35], 0.26666666666666666, Ops::fmac(KL[32], 0.13333333333333333, Ops::fmac(KL[31], 0.13333333333333333, Ops::fmac(KL[30], 0.13333333333333333, Ops::fmac(KL[25], 0.26666666666666666, Ops::fmac(KL[22], 0.13333333333333333, Ops::fmac(KL[21], 0.26666666666666666, Ops::fmac(KL[20], 0.26666666666666666, Ops::fmac(KL[15], 0.26666666666666666, Ops::fmac(KL[12], 0.26666666666666666, Ops::fmac(KL[11], 0.13333333333333333, Ops::fmac(KL[10], 0.26666666666666666, Ops::fmac(KL[5], 0.8, Ops::fmac(KL[2], 0.26666666666666666, Ops::fmac(KL[1], 0.26666666666666666, Ops::mulc(KL[0], 0.13333333333333333))))))))))))))));
    K[36] = Ops::fmac(KL[36], 0.26666666666666666, Ops::fmac(KL[33], 0.13333333333333333, Ops::fmac(KL[31], 0.26666666666666666, Ops::fmac(KL[30], 0.26666666666666666, Ops::fmac(KL[26], 0.26666666666666666, Ops::fmac(KL[23], 0.13333333333333333, Ops::fmac(KL[21], 0.13333333333333333, Ops::fmac(KL[20], 0.13333333333333333, Ops::fmac(KL[16], 0.26666666666666666, Ops::fmac(KL[13], 0.26666666666666666, Ops::fmac(KL[11], 0.13333333333333333, Ops::fmac(KL[10], 0.26666666666666666, Ops::fmac(KL[6], 0.8, Ops::fmac(KL[3], 0.26666666666666666, Ops::fmac(KL[1], 0.26666666666666666, Ops::mulc(KL[0], 0.13333333333333333))))))))))))))));
    K[37] = Ops::fmac(KL[35], 0.13333333333333333, Ops::fmac(KL[34], 0.13333333333333333, Ops::fmac(KL[32], 0.26666666666666666, Ops::fmac(KL[31], 0.13333333333333333, Ops::fmac(KL[25], 0.13333333333333333, Ops::fmac(KL[24], 0.26666666666666666, Ops::fmac(KL[22], 0.26666666666666666, Ops::fmac(KL[21], 0.26666666666666666, Ops::fmac(KL[15], 0.26666666666666666, Ops::fmac(KL[14], 0.13333333333333333, Ops::fmac(KL[12], 0.8, Ops::fmac(KL[11], 0.26666666666666666, Ops::fmac(KL[5], 0.26666666666666666, Ops::fmac(KL[4], 0.26666666666666666, Ops::fmac(KL[2], 0.26666666666666666, Ops::mulc(KL[1], 0.13333333333333333))))))))))))))));
    K[38] = Ops::fmac(KL[36], 0.13333333333333333, Ops::fmac(KL[34], 0.26666666666666666, Ops::fmac(KL[33], 0.26666666666666666, Ops::fmac(KL[31], 0.26666666666666666, Ops::fmac(KL[26], 0.13333333333333333, Ops::fmac(KL[24], 0.13333333333333333, Ops::fmac(KL[23], 0.26666666666666666, Ops::fmac(KL[21], 0.13333333333333333, Ops::fmac(KL[16], 0.26666666666666666, Ops::fmac(KL[14], 0.13333333333333333, Ops::fmac(KL[13], 0.8, Ops::fmac(KL[11], 0.26666666666666666, Ops::fmac(KL[6], 0.26666666666666666, Ops::fmac(KL[4], 0.26666666666666666, Ops::fmac(KL[3], 0.26666666666666666, Ops::mulc(KL[1], 0.13333333333333333))))))))))))))));
    K[39] = Ops::fmac(KL[36], 0.13333333333333333, Ops::fmac(KL[35], 0.26666666666666666, Ops::fmac(KL[33], 0.13333333333333333, Ops::fmac(KL[32], 0.26666666666666666, Ops::fmac(KL[26], 0.26666666666666666, Ops::fmac(KL[25], 0.13333333333333333, Ops::fmac(KL[23], 0.26666666666666666, Ops::fmac(KL[22], 0.13333333333333333, Ops::fmac(KL[16], 0.13333333333333333, Ops::fmac(KL[15], 0.13333333333333333, Ops::fmac(KL[13], 0.26666666666666666, Ops::fmac(KL[12], 0.26666666666666666, Ops::fmac(KL[6], 0.26666666666666666, Ops::fmac(KL[5], 0.26666666666666666, Ops::fmac(KL[3], 0.13333333333333333, Ops::mulc(KL[2], 0.13333333333333333))))))))))))))));
    K[40] = Ops::fmac(KL[37], 0.26666666666666666, Ops::fmac(KL[32], 0.26666666666666666, Ops::fmac(KL[30], 0.26666666666666666, Ops::fmac(KL[27], 0.26666666666666666, Ops::fmac(KL[22], 0.5333333333333333, Ops::fmac(KL[20], 0.8, Ops::fmac(KL[17], 0.26666666666666666, Ops::fmac(KL[12], 0.26666666666666666, Ops::fmac(KL[10], 0.26666666666666666, Ops::fmac(KL[7], 0.8, Ops::fmac(KL[2], 0.5333333333333333, Ops::mulc(KL[0], 0.26666666666666666))))))))))));
    K[41] = Ops::fmac(KL[38], 0.26666666666666666, Ops::fmac(KL[33], 0.13333333333333333, Ops::fmac(KL[32], 0.26666666666666666, Ops::fmac(KL[30], 0.26666666666666666, Ops::fmac(KL[28], 0.26666666666666666, Ops::fmac(KL[23], 0.26666666666666666, Ops::fmac(KL[22], 0.13333333333333333, Ops::fmac(KL[20], 0.26666666666666666, Ops::fmac(KL[18], 0.26666666666666666, Ops::fmac(KL[13], 0.13333333333333333, Ops::fmac(KL[12], 0.13333333333333333, Ops::fmac(KL[10], 0.13333333333333333, Ops::fmac(KL[8], 0.8, Ops::fmac(KL[3], 0.26666666666666666, Ops::fmac(KL[2], 0.26666666666666666, Ops::mulc(KL[0], 0.13333333333333333))))))))))))))));
    K[42] = Ops::fmac(KL[37], 0.13333333333333333, Ops::fmac(KL[35], 0.13333333333333333, Ops::fmac(KL[32], 0.13333333333333333, Ops::fmac(KL[31], 0.26666666666666666, Ops::fmac(KL[27], 0.13333333333333333, Ops::fmac(KL[25], 0.26666666666666666, Ops::fmac(KL[22], 0.26666666666666666, Ops::fmac(KL[21], 0.8, Ops::fmac(KL[17], 0.26666666666666666, Ops::fmac(KL[15], 0.13333333333333333, Ops::fmac(KL[12], 0.26666666666666666, Ops::fmac(KL[11], 0.26666666666666666, Ops::fmac(KL[7], 0.26666666666666666, Ops::fmac(KL[5], 0.26666666666666666, Ops::fmac(KL[2], 0.13333333333333333, Ops::mulc(KL[1], 0.26666666666666666))))))))))))))));
    K[43] = Ops::fmac(KL[38], 0.13333333333333333, Ops::fmac(KL[35], 0.26666666666666666, Ops::fmac(KL[33], 0.13333333333333333, Ops::fmac(KL[31], 0.26666666666666666, Ops::fmac(KL[28], 0.13333333333333333, Ops::fmac(KL[25], 0.13333333333333333, Ops::fmac(KL[23], 0.26666666666666666, Ops::fmac(KL[21], 0.26666666666666666, Ops::fmac(KL[18], 0.26666666666666666, Ops::fmac(KL[15], 0.13333333333333333, Ops::fmac(KL[13], 0.26666666666666666, Ops::fmac(KL[11], 0.13333333333333333, Ops::fmac(KL[8], 0.26666666666666666, Ops::fmac(KL[5], 0.26666666666666666, Ops::fmac(KL[3], 0.13333333333333333, Ops::mulc(KL[1], 0.13333333333333333))))))))))))))));
    K[44] = Ops::fmac(KL[38], 0.13333333333333333, Ops::fmac(KL[37], 0.26666666666666666, Ops::fmac(KL[33], 0.26666666666666666, Ops::fmac(KL[32], 0.26666666666666666, Ops::fmac(KL[28], 0.26666666666666666, Ops::fmac(KL[27], 0.13333333333333333, Ops::fmac(KL[23], 0.8, Ops::fmac(KL[22], 0.26666666666666666, Ops::fmac(KL[18], 0.13333333333333333, Ops::fmac(KL[17], 0.13333333333333333, Ops::fmac(KL[13], 0.26666666666666666, Ops::fmac(KL[12], 0.13333333333333333, Ops::fmac(KL[8], 0.26666666666666666, Ops::fmac(KL[7], 0.26666666666666666, Ops::fmac(KL[3], 0.26666666666666666, Ops::mulc(KL[2], 0.13333333333333333))))))))))))))));
    K[45] = Ops::fmac(KL[39], 0.26666666666666666, Ops::fmac(KL[33], 0.5333333333333333, Ops::fmac(KL[30], 0.8, Ops::fmac(KL[29], 0.26666666666666666, Ops::fmac(KL[23], 0.26666666666666666, Ops::fmac(KL[20], 0.26666666666666666, Ops::fmac(KL[19], 0.26666666666666666, Ops::fmac(KL[13], 0.26666666666666666, Ops::fmac(KL[10], 0.26666666666666666, Ops::fmac(KL[9], 0.8, Ops::fmac(KL[3], 0.5333333333333333, Ops::mulc(KL[0], 0.26666666666666666))))))))))));
    K[46] = Ops::fmac(KL[38], 0.13333333333333333, Ops::fmac(KL[36], 0.13333333333333333, Ops::fmac(KL[32], 0.26666666666666666, Ops::fmac(KL[31], 0.26666666666666666, Ops::fmac(KL[28], 0.13333333333333333, Ops::fmac(KL[26], 0.26666666666666666, Ops::fmac(KL[22], 0.13333333333333333, Ops::fmac(KL[21], 0.26666666666666666, Ops::fmac(KL[18], 0.26666666666666666, Ops::fmac(KL[16], 0.13333333333333333, Ops::fmac(KL[12], 0.26666666666666666, Ops::fmac(KL[11], 0.13333333333333333, Ops::fmac(KL[8], 0.26666666666666666, Ops::fmac(KL[6], 0.26666666666666666, Ops::fmac(KL[2], 0.13333333333333333, Ops::mulc(KL[1], 0.13333333333333333))))))))))))))));
    K[47] = Ops::fmac(KL[39], 0.13333333333333333, Ops::fmac(KL[36], 0.26666666666666666, Ops::fmac(KL[33], 0.26666666666666666, Ops::fmac(KL[31], 0.8, Ops::fmac(KL[29], 0.13333333333333333, Ops::fmac(KL[26], 0.13333333333333333, Ops::fmac(KL[23], 0.13333333333333333, Ops::fmac(KL[21], 0.26666666666666666, Ops::fmac(KL[19], 0.26666666666666666, Ops::fmac(KL[16], 0.13333333333333333, Ops::fmac(KL[13], 0.26666666666666666, Ops::fmac(KL[11], 0.26666666666666666, Ops::fmac(KL[9], 0.26666666666666666, Ops::fmac(KL[6], 0.26666666666666666, Ops::fmac(KL[3], 0.13333333333333333, Ops::mulc(KL[1], 0.26666666666666666))))))))))))))));
    K[48] = Ops::fmac(KL[39], 0.13333333333333333, Ops::fmac(KL[38], 0.26666666666666666, Ops::fmac(KL[33], 0.26666666666666666, Ops::fmac(KL[32], 0.8, Ops::fmac(KL[29], 0.26666666666666666, Ops::fmac(KL[28], 0.13333333333333333, Ops::fmac(KL[23], 0.26666666666666666, Ops::fmac(KL[22], 0.26666666666666666, Ops::fmac(KL[19], 0.13333333333333333, Ops::fmac(KL[18], 0.13333333333333333, Ops::fmac(KL[13], 0.13333333333333333, Ops::fmac(KL[12], 0.26666666666666666, Ops::fmac(KL[9], 0.26666666666666666, Ops::fmac(KL[8], 0.26666666666666666, Ops::fmac(KL[3], 0.13333333333333333, Ops::mulc(KL[2], 0.26666666666666666))))))))))))))));
    K[49] = Ops::fmac(KL[37], 0.26666666666666666, Ops::fmac(KL[35], 0.26666666666666666, Ops::fmac(KL[34], 0.26666666666666666, Ops::fmac(KL[27], 0.26666666666666666, Ops::fmac(KL[25], 0.5333333333333333, Ops::fmac(KL[24], 0.8, Ops::fmac(KL[17], 0.8, Ops::fmac(KL[15], 0.5333333333333333, Ops::fmac(KL[14], 0.26666666666666666, Ops::fmac(KL[7], 0.26666666666666666, Ops::fmac(KL[5], 0.26666666666666666, Ops::mulc(KL[4], 0.26666666666666666))))))))))));
    K[50] = Ops::fmac(KL[38], 0.26666666666666666, Ops::fmac(KL[36], 0.13333333333333333, Ops::fmac(KL[35], 0.26666666666666666, Ops::fmac(KL[34], 0.26666666666666666, Ops::fmac(KL[28], 0.26666666666666666, Ops::fmac(KL[26], 0.26666666666666666, Ops::fmac(KL[25], 0.13333333333333333, Ops::fmac(KL[24], 0.26666666666666666, Ops::fmac(KL[18], 0.8, Ops::fmac(KL[16], 0.26666666666666666, Ops::fmac(KL[15], 0.26666666666666666, Ops::fmac(KL[14], 0.13333333333333333, Ops::fmac(KL[8], 0.26666666666666666, Ops::fmac(KL[6], 0.13333333333333333, Ops::fmac(KL[5], 0.13333333333333333, Ops::mulc(KL[4], 0.13333333333333333))))))))))))))));
    K[51] = Ops::fmac(KL[38], 0.13333333333333333, Ops::fmac(KL[37], 0.26666666666666666, Ops::fmac(KL[36], 0.26666666666666666, Ops::fmac(KL[35], 0.26666666666666666, Ops::fmac(KL[28], 0.26666666666666666, Ops::fmac(KL[27], 0.13333333333333333, Ops::fmac(KL[26], 0.8, Ops::fmac(KL[25], 0.26666666666666666, Ops::fmac(KL[18], 0.26666666666666666, Ops::fmac(KL[17], 0.26666666666666666, Ops::fmac(KL[16], 0.26666666666666666, Ops::fmac(KL[15], 0.13333333333333333, Ops::fmac(KL[8], 0.13333333333333333, Ops::fmac(KL[7], 0.13333333333333333, Ops::fmac(KL[6], 0.26666666666666666, Ops::mulc(KL[5], 0.13333333333333333))))))))))))))));
    K[52] = Ops::fmac(KL[39], 0.26666666666666666, Ops::fmac(KL[36], 0.5333333333333333, Ops::fmac(KL[34], 0.8, Ops::fmac(KL[29], 0.26666666666666666, Ops::fmac(KL[26], 0.26666666666666666, Ops::fmac(KL[24], 0.26666666666666666, Ops::fmac(KL[19], 0.8, Ops::fmac(KL[16], 0.5333333333333333, Ops::fmac(KL[14], 0.26666666666666666, Ops::fmac(KL[9], 0.26666666666666666, Ops::fmac(KL[6], 0.26666666666666666, Ops::mulc(KL[4], 0.26666666666666666))))))))))));
    K[53] = Ops::fmac(KL[39], 0.13333333333333333, Ops::fmac(KL[38], 0.26666666666666666, Ops::fmac(KL[36], 0.26666666666666666, Ops::fmac(KL[35], 0.8, Ops::fmac(KL[29], 0.26666666666666666, Ops::fmac(KL[28], 0.13333333333333333, Ops::fmac(KL[26], 0.26666666666666666, Ops::fmac(KL[25], 0.26666666666666666, Ops::fmac(KL[19], 0.26666666666666666, Ops::fmac(KL[18], 0.26666666666666666, Ops::fmac(KL[16], 0.13333333333333333, Ops::fmac(KL[15], 0.26666666666666666, Ops::fmac(KL[9], 0.13333333333333333, Ops::fmac(KL[8], 0.13333333333333333, Ops::fmac(KL[6], 0.13333333333333333, Ops::mulc(KL[5], 0.26666666666666666))))))))))))))));
    K[54] = Ops::fmac(KL[39], 0.26666666666666666, Ops::fmac(KL[38], 0.5333333333333333, Ops::fmac(KL[37], 0.8, Ops::fmac(KL[29], 0.8, Ops::fmac(KL[28], 0.5333333333333333, Ops::fmac(KL[27], 0.26666666666666666, Ops::fmac(KL[19], 0.26666666666666666, Ops::fmac(KL[18], 0.26666666666666666, Ops::fmac(KL[17], 0.26666666666666666, Ops::fmac(KL[9], 0.26666666666666666, Ops::fmac(KL[8], 0.26666666666666666, Ops::mulc(KL[7], 0.26666666666666666))))))))))));
  }
  static constexpr int TERMS = 544;
};

template <> struct KappaTC<2, 4> {
  static constexpr int N = 120, K = 18, ND = 15;
};
#ifdef FE_GEN_KAPPA_TC_TABLES
// row n: upper-triangle pair (I[n], J[n]); column k = kappa node * 6 + Lam pair
static __constant__ unsigned char kKappaTC24_I[120] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 2, 2, 2, 2, 2, 2, 2, 2, 2, 2, 2, 2, 2, 3, 3, 3, 3, 3, 3, 3, 3, 3, 3, 3, 3, 4, 4, 4, 4, 4, 4, 4, 4, 4, 4, 4, 5, 5, 5, 5, 5, 5, 5, 5, 5, 5, 6, 6, 6, 6, 6, 6, 6, 6, 6, 7, 7, 7, 7, 7, 7, 7, 7, 8, 8, 8, 8, 8, 8, 8, 9, 9, 9, 9, 9, 9, 10, 10, 10, 10, 10, 11, 11, 11, 11, 12, 12, 12, 13, 13, 14};
static __constant__ unsigned char kKappaTC24_J[120] = {0, 1, 2, 3, 4, 5, 6, 7, 8, 9, 10, 11, 12, 13, 14, 1, 2, 3, 4, 5, 6, 7, 8, 9, 10, 11, 12, 13, 14, 2, 3, 4, 5, 6, 7, 8, 9, 10, 11, 12, 13, 14, 3, 4, 5, 6, 7, 8, 9, 10, 11, 12, 13, 14, 4, 5, 6, 7, 8, 9, 10, 11, 12, 13, 14, 5, 6, 7, 8, 9, 10, 11, 12, 13, 14, 6, 7, 8, 9, 10, 11, 12, 13, 14, 7, 8, 9, 10, 11, 12, 13, 14, 8, 9, 10, 11, 12, 13, 14, 9, 10, 11, 12, 13, 14, 10, 11, 12, 13, 14, 11, 12, 13, 14, 12, 13, 14, 13, 14, 14};
static __device__ const float kKappaTC24_C[120][18] = {{0.5943562388420105f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.07583773881196976f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.07583773881196976f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f},
    {0.0f, -0.05149911716580391f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f, -0.05149911716580391f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f, -0.010229276493191719f, 0.0f, 0.0f, 0.0f, 0.0f},
    {0.0f, 0.0f, -0.05149911716580391f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f, -0.010229276493191719f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f, -0.05149911716580391f, 0.0f, 0.0f, 0.0f},
    {0.4021163880825043f, 1.3742504119873047f, 0.0f, 0.0f, 0.0f, 0.0f, -0.09876543283462524f, 0.09171076118946075f, 0.0f, 0.0f, 0.0f, 0.0f, -0.04938271641731262f, 0.09171076118946075f, 0.0f, 0.0f, 0.0f, 0.0f},
    {-0.1358024626970291f, -0.7343915104866028f, 0.0f, 0.0f, 0.0f, 0.0f, 0.17989417910575867f, -0.051146384328603745f, 0.0f, 0.0f, 0.0f, 0.0f, 0.04056437313556671f, -0.06525573134422302f, 0.0f, 0.0f, 0.0f, 0.0f},
    {0.035273369401693344f, 0.3075837790966034f, 0.0f, 0.0f, 0.0f, 0.0f, -0.10440917313098907f, 0.0634920671582222f, 0.0f, 0.0f, 0.0f, 0.0f, -0.015520282089710236f, 0.035273369401693344f, 0.0f, 0.0f, 0.0f, 0.0f},
    {0.4021163880825043f, 0.0f, 1.3742504119873047f, 0.0f, 0.0f, 0.0f, -0.04938271641731262f, 0.0f, 0.09171076118946075f, 0.0f, 0.0f, 0.0f, -0.09876543283462524f, 0.0f, 0.09171076118946075f, 0.0f, 0.0f, 0.0f},
    {-0.1358024626970291f, 0.0f, -0.7343915104866028f, 0.0f, 0.0f, 0.0f, 0.04056437313556671f, 0.0f, -0.06525573134422302f, 0.0f, 0.0f, 0.0f, 0.17989417910575867f, 0.0f, -0.051146384328603745f, 0.0f, 0.0f, 0.0f},
    {0.035273369401693344f, 0.0f, 0.3075837790966034f, 0.0f, 0.0f, 0.0f, -0.015520282089710236f, 0.0f, 0.035273369401693344f, 0.0f, 0.0f, 0.0f, -0.10440917313098907f, 0.0f, 0.0634920671582222f, 0.0f, 0.0f, 0.0f},
    {0.0f, 0.035273369401693344f, 0.035273369401693344f, 0.0f, 0.0f, 0.0f, 0.0f, -0.08888889104127884f, -0.10440917313098907f, 0.0f, 0.0f, 0.0f, 0.0f, -0.03104056417942047f, -0.015520282089710236f, 0.0f, 0.0f, 0.0f},
    {0.0f, 0.019400352612137794f, 0.019400352612137794f, 0.0f, 0.0f, 0.0f, 0.0f, -0.04691357910633087f, -0.05714285746216774f, 0.0f, 0.0f, 0.0f, 0.0f, -0.05714285746216774f, -0.04691357910633087f, 0.0f, 0.0f, 0.0f},
    {0.0f, 0.035273369401693344f, 0.035273369401693344f, 0.0f, 0.0f, 0.0f, 0.0f, -0.015520282089710236f, -0.03104056417942047f, 0.0f, 0.0f, 0.0f, 0.0f, -0.10440917313098907f, -0.08888889104127884f, 0.0f, 0.0f, 0.0f},
    {0.07054673880338669f, 0.5925925970077515f, 0.5925925970077515f, 0.0f, 0.0f, 0.0f, 0.1975308656692505f, 0.014109347015619278f, 0.028218694031238556f, 0.0f, 0.0f, 0.0f, 0.1975308656692505f, 0.028218694031238556f, 0.014109347015619278f, 0.0f, 0.0f, 0.0f},
    {0.014109347015619278f, -0.14109347760677338f, -0.14109347760677338f, 0.0f, 0.0f, 0.0f, -0.15238095819950104f, 0.07054673880338669f, 0.08465608209371567f, 0.0f, 0.0f, 0.0f, -0.0733686089515686f, 0.028218694031238556f, 0.014109347015619278f, 0.0f, 0.0f, 0.0f},
    {0.014109347015619278f, -0.14109347760677338f, -0.14109347760677338f, 0.0f, 0.0f, 0.0f, -0.0733686089515686f, 0.014109347015619278f, 0.028218694031238556f, 0.0f, 0.0f, 0.0f, -0.15238095819950104f, 0.08465608209371567f, 0.07054673880338669f, 0.0f, 0.0f, 0.0f},
    {0.0f, 0.0f, 0.0f, 0.07583773881196976f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.5943562388420105f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.07583773881196976f, 0.0f, 0.0f},
    {0.0f, 0.0f, 0.0f, 0.0f, -0.010229276493191719f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f, -0.05149911716580391f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f, -0.05149911716580391f, 0.0f},
    {0.0f, 0.0634920671582222f, 0.0f, -0.10440917313098907f, 0.0f, 0.0f, 0.0f, 0.3075837790966034f, 0.0f, 0.035273369401693344f, 0.0f, 0.0f, 0.0f, 0.035273369401693344f, 0.0f, -0.015520282089710236f, 0.0f, 0.0f},
    {0.0f, -0.051146384328603745f, 0.0f, 0.17989417910575867f, 0.0f, 0.0f, 0.0f, -0.7343915104866028f, 0.0f, -0.1358024626970291f, 0.0f, 0.0f, 0.0f, -0.06525573134422302f, 0.0f, 0.04056437313556671f, 0.0f, 0.0f},
    {0.0f, 0.09171076118946075f, 0.0f, -0.09876543283462524f, 0.0f, 0.0f, 0.0f, 1.3742504119873047f, 0.0f, 0.4021163880825043f, 0.0f, 0.0f, 0.0f, 0.09171076118946075f, 0.0f, -0.04938271641731262f, 0.0f, 0.0f},
    {0.0f, -0.08888889104127884f, 0.0f, 0.0f, -0.10440917313098907f, 0.0f, 0.0f, 0.035273369401693344f, 0.0f, 0.0f, 0.035273369401693344f, 0.0f, 0.0f, -0.03104056417942047f, 0.0f, 0.0f, -0.015520282089710236f, 0.0f},
    {0.0f, -0.04691357910633087f, 0.0f, 0.0f, -0.05714285746216774f, 0.0f, 0.0f, 0.019400352612137794f, 0.0f, 0.0f, 0.019400352612137794f, 0.0f, 0.0f, -0.05714285746216774f, 0.0f, 0.0f, -0.04691357910633087f, 0.0f},
    {0.0f, -0.015520282089710236f, 0.0f, 0.0f, -0.03104056417942047f, 0.0f, 0.0f, 0.035273369401693344f, 0.0f, 0.0f, 0.035273369401693344f, 0.0f, 0.0f, -0.10440917313098907f, 0.0f, 0.0f, -0.08888889104127884f, 0.0f},
    {0.0f, 0.0f, 0.0f, -0.04938271641731262f, 0.09171076118946075f, 0.0f, 0.0f, 0.0f, 0.0f, 0.4021163880825043f, 1.3742504119873047f, 0.0f, 0.0f, 0.0f, 0.0f, -0.09876543283462524f, 0.09171076118946075f, 0.0f},
    {0.0f, 0.0f, 0.0f, 0.04056437313556671f, -0.06525573134422302f, 0.0f, 0.0f, 0.0f, 0.0f, -0.1358024626970291f, -0.7343915104866028f, 0.0f, 0.0f, 0.0f, 0.0f, 0.17989417910575867f, -0.051146384328603745f, 0.0f},
    {0.0f, 0.0f, 0.0f, -0.015520282089710236f, 0.035273369401693344f, 0.0f, 0.0f, 0.0f, 0.0f, 0.035273369401693344f, 0.3075837790966034f, 0.0f, 0.0f, 0.0f, 0.0f, -0.10440917313098907f, 0.0634920671582222f, 0.0f},
    {0.0f, 0.07054673880338669f, 0.0f, -0.15238095819950104f, 0.08465608209371567f, 0.0f, 0.0f, -0.14109347760677338f, 0.0f, 0.014109347015619278f, -0.14109347760677338f, 0.0f, 0.0f, 0.028218694031238556f, 0.0f, -0.0733686089515686f, 0.014109347015619278f, 0.0f},
    {0.0f, 0.014109347015619278f, 0.0f, 0.1975308656692505f, 0.028218694031238556f, 0.0f, 0.0f, 0.5925925970077515f, 0.0f, 0.07054673880338669f, 0.5925925970077515f, 0.0f, 0.0f, 0.028218694031238556f, 0.0f, 0.1975308656692505f, 0.014109347015619278f, 0.0f},
    {0.0f, 0.014109347015619278f, 0.0f, -0.0733686089515686f, 0.028218694031238556f, 0.0f, 0.0f, -0.14109347760677338f, 0.0f, 0.014109347015619278f, -0.14109347760677338f, 0.0f, 0.0f, 0.08465608209371567f, 0.0f, -0.15238095819950104f, 0.07054673880338669f, 0.0f},
    {0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.07583773881196976f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.07583773881196976f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.5943562388420105f},
    {0.0f, 0.0f, -0.08888889104127884f, 0.0f, -0.10440917313098907f, 0.0f, 0.0f, 0.0f, -0.03104056417942047f, 0.0f, -0.015520282089710236f, 0.0f, 0.0f, 0.0f, 0.035273369401693344f, 0.0f, 0.035273369401693344f, 0.0f},
    {0.0f, 0.0f, -0.04691357910633087f, 0.0f, -0.05714285746216774f, 0.0f, 0.0f, 0.0f, -0.05714285746216774f, 0.0f, -0.04691357910633087f, 0.0f, 0.0f, 0.0f, 0.019400352612137794f, 0.0f, 0.019400352612137794f, 0.0f},
    {0.0f, 0.0f, -0.015520282089710236f, 0.0f, -0.03104056417942047f, 0.0f, 0.0f, 0.0f, -0.10440917313098907f, 0.0f, -0.08888889104127884f, 0.0f, 0.0f, 0.0f, 0.035273369401693344f, 0.0f, 0.035273369401693344f, 0.0f},
    {0.0f, 0.0f, 0.0634920671582222f, 0.0f, 0.0f, -0.10440917313098907f, 0.0f, 0.0f, 0.035273369401693344f, 0.0f, 0.0f, -0.015520282089710236f, 0.0f, 0.0f, 0.3075837790966034f, 0.0f, 0.0f, 0.035273369401693344f},
    {0.0f, 0.0f, -0.051146384328603745f, 0.0f, 0.0f, 0.17989417910575867f, 0.0f, 0.0f, -0.06525573134422302f, 0.0f, 0.0f, 0.04056437313556671f, 0.0f, 0.0f, -0.7343915104866028f, 0.0f, 0.0f, -0.1358024626970291f},
    {0.0f, 0.0f, 0.09171076118946075f, 0.0f, 0.0f, -0.09876543283462524f, 0.0f, 0.0f, 0.09171076118946075f, 0.0f, 0.0f, -0.04938271641731262f, 0.0f, 0.0f, 1.3742504119873047f, 0.0f, 0.0f, 0.4021163880825043f},
    {0.0f, 0.0f, 0.0f, 0.0f, 0.035273369401693344f, -0.015520282089710236f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0634920671582222f, -0.10440917313098907f, 0.0f, 0.0f, 0.0f, 0.0f, 0.3075837790966034f, 0.035273369401693344f},
    {0.0f, 0.0f, 0.0f, 0.0f, -0.06525573134422302f, 0.04056437313556671f, 0.0f, 0.0f, 0.0f, 0.0f, -0.051146384328603745f, 0.17989417910575867f, 0.0f, 0.0f, 0.0f, 0.0f, -0.7343915104866028f, -0.1358024626970291f},
    {0.0f, 0.0f, 0.0f, 0.0f, 0.09171076118946075f, -0.04938271641731262f, 0.0f, 0.0f, 0.0f, 0.0f, 0.09171076118946075f, -0.09876543283462524f, 0.0f, 0.0f, 0.0f, 0.0f, 1.3742504119873047f, 0.4021163880825043f},
    {0.0f, 0.0f, 0.07054673880338669f, 0.0f, 0.08465608209371567f, -0.15238095819950104f, 0.0f, 0.0f, 0.028218694031238556f, 0.0f, 0.014109347015619278f, -0.0733686089515686f, 0.0f, 0.0f, -0.14109347760677338f, 0.0f, -0.14109347760677338f, 0.014109347015619278f},
    {0.0f, 0.0f, 0.014109347015619278f, 0.0f, 0.028218694031238556f, -0.0733686089515686f, 0.0f, 0.0f, 0.08465608209371567f, 0.0f, 0.07054673880338669f, -0.15238095819950104f, 0.0f, 0.0f, -0.14109347760677338f, 0.0f, -0.14109347760677338f, 0.014109347015619278f},
    {0.0f, 0.0f, 0.014109347015619278f, 0.0f, 0.028218694031238556f, 0.1975308656692505f, 0.0f, 0.0f, 0.028218694031238556f, 0.0f, 0.014109347015619278f, 0.1975308656692505f, 0.0f, 0.0f, 0.5925925970077515f, 0.0f, 0.5925925970077515f, 0.07054673880338669f},
    {2.0317461490631104f, 3.250793695449829f, 0.0f, 3.566843032836914f, 0.0f, 0.0f, 1.2190476655960083f, 0.6320987939834595f, 0.0f, 0.31604939699172974f, 0.0f, 0.0f, 0.40634921193122864f, 0.31604939699172974f, 0.0f, 0.31604939699172974f, 0.0f, 0.0f},
    {-0.16931216418743134f, 0.5530864000320435f, 0.0f, -1.388359785079956f, 0.0f, 0.0f, -0.9142857193946838f, 0.4740740656852722f, 0.0f, 0.04514991119503975f, 0.0f, 0.0f, -0.2370370328426361f, 0.022574955597519875f, 0.0f, -0.180599644780159f, 0.0f, 0.0f},
    {0.0f, -0.31604939699172974f, 0.0f, 0.5869488716125488f, 0.0f, 0.0f, 0.5869488716125488f, -0.31604939699172974f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0902998223900795f, -0.04514991119503975f, 0.0f, 0.0902998223900795f, 0.0f, 0.0f},
    {1.0158730745315552f, 1.6253968477249146f, 1.6253968477249146f, 0.0f, 3.566843032836914f, 0.0f, 0.40634921193122864f, 0.15802469849586487f, 0.31604939699172974f, 0.0f, 0.31604939699172974f, 0.0f, 0.40634921193122864f, 0.31604939699172974f, 0.15802469849586487f, 0.0f, 0.31604939699172974f, 0.0f},
    {-0.3216931223869324f, -0.42892417311668396f, -0.7788359522819519f, 0.0f, -1.388359785079956f, 0.0f, -0.16931216418743134f, -0.06208112835884094f, -0.2370370328426361f, 0.0f, -0.180599644780159f, 0.0f, -0.2370370328426361f, -0.10158730298280716f, 0.08465608209371567f, 0.0f, 0.04514991119503975f, 0.0f},
    {0.06772486865520477f, 0.0902998223900795f, 0.40634921193122864f, 0.0f, 0.5869488716125488f, 0.0f, 0.04514991119503975f, 0.022574955597519875f, 0.13544973731040955f, 0.0f, 0.0902998223900795f, 0.0f, 0.0902998223900795f, 0.0902998223900795f, -0.06772486865520477f, 0.0f, 0.0f, 0.0f},
    {0.0f, -0.06772486865520477f, 0.0f, 0.0902998223900795f, 0.0902998223900795f, 0.0f, 0.0f, 0.40634921193122864f, 0.5869488716125488f, 0.06772486865520477f, 0.0902998223900795f, 0.0f, 0.0f, 0.13544973731040955f, 0.0902998223900795f, 0.04514991119503975f, 0.022574955597519875f, 0.0f},
    {0.0f, -0.05079365149140358f, -0.033862434327602386f, 0.022574955597519875f, 0.022574955597519875f, 0.0f, 0.0f, 0.10158730298280716f, 0.16931216418743134f, 0.028218694031238556f, 0.033862434327602386f, 0.0f, 0.0f, 0.16931216418743134f, 0.16931216418743134f, 0.033862434327602386f, 0.028218694031238556f, 0.0f},
    {0.0f, 0.06772486865520477f, 0.13544973731040955f, 0.0902998223900795f, 0.0902998223900795f, 0.0f, 0.0f, 0.04514991119503975f, 0.13544973731040955f, 0.022574955597519875f, 0.04514991119503975f, 0.0f, 0.0f, 0.0902998223900795f, 0.13544973731040955f, 0.0902998223900795f, 0.06772486865520477f, 0.0f},
    {0.9481481313705444f, 2.3477954864501953f, 3.521693229675293f, 2.573544979095459f, 2.573544979095459f, 0.0f, -0.40634921193122864f, 0.4514991044998169f, 1.2190476655960083f, 0.22574955224990845f, 0.4514991044998169f, 0.0f, -0.2708994746208191f, 0.4514991044998169f, 0.40634921193122864f, 0.4514991044998169f, 0.22574955224990845f, 0.0f},
    {-0.13544973731040955f, 0.0902998223900795f, -0.2708994746208191f, -0.49664902687072754f, -0.49664902687072754f, 0.0f, 0.6772486567497253f, 0.0f, -0.40634921193122864f, 0.04514991119503975f, 0.0f, 0.0f, 0.2708994746208191f, -0.0902998223900795f, -0.13544973731040955f, -0.0902998223900795f, -0.04514991119503975f, 0.0f},
    {-0.13544973731040955f, -0.4514991044998169f, -0.8126984238624573f, -0.49664902687072754f, -0.49664902687072754f, 0.0f, 0.13544973731040955f, -0.0902998223900795f, -0.40634921193122864f, -0.04514991119503975f, -0.0902998223900795f, 0.0f, 0.2708994746208191f, 0.0f, -0.13544973731040955f, 0.0f, 0.04514991119503975f, 0.0f},
    {1.244444489479065f, 1.7777777910232544f, 0.0f, 3.1576719284057617f, 0.0f, 0.0f, 3.1576719284057617f, 1.7777777910232544f, 0.0f, 1.244444489479065f, 0.0f, 0.0f, 0.49947088956832886f, 0.3301587402820587f, 0.0f, 0.49947088956832886f, 0.0f, 0.0f},
    {0.04514991119503975f, 0.4740740656852722f, 0.0f, -0.9142857193946838f, 0.0f, 0.0f, -1.388359785079956f, 0.5530864000320435f, 0.0f, -0.16931216418743134f, 0.0f, 0.0f, -0.180599644780159f, 0.022574955597519875f, 0.0f, -0.2370370328426361f, 0.0f, 0.0f},
    {-0.3216931223869324f, -0.7788359522819519f, -0.42892417311668396f, 0.0f, -1.388359785079956f, 0.0f, -0.2370370328426361f, 0.08465608209371567f, -0.10158730298280716f, 0.0f, 0.04514991119503975f, 0.0f, -0.16931216418743134f, -0.2370370328426361f, -0.06208112835884094f, 0.0f, -0.180599644780159f, 0.0f},
    {-0.10582010447978973f, -0.1608465611934662f, -0.1608465611934662f, 0.0f, -0.3640211522579193f, 0.0f, -0.09312169253826141f, -0.10582010447978973f, -0.1269841343164444f, 0.0f, -0.21164020895957947f, 0.0f, -0.09312169253826141f, -0.1269841343164444f, -0.10582010447978973f, 0.0f, -0.21164020895957947f, 0.0f},
    {0.028218694031238556f, 0.033862434327602386f, 0.10158730298280716f, 0.0f, 0.16931216418743134f, 0.0f, 0.033862434327602386f, 0.028218694031238556f, 0.16931216418743134f, 0.0f, 0.16931216418743134f, 0.0f, 0.022574955597519875f, 0.022574955597519875f, -0.05079365149140358f, 0.0f, -0.033862434327602386f, 0.0f},
    {0.0f, 0.08465608209371567f, 0.04514991119503975f, -0.2370370328426361f, -0.10158730298280716f, 0.0f, 0.0f, -0.7788359522819519f, -1.388359785079956f, -0.3216931223869324f, -0.42892417311668396f, 0.0f, 0.0f, -0.2370370328426361f, -0.180599644780159f, -0.16931216418743134f, -0.06208112835884094f, 0.0f},
    {0.0f, -0.10582010447978973f, -0.21164020895957947f, -0.09312169253826141f, -0.1269841343164444f, 0.0f, 0.0f, -0.1608465611934662f, -0.3640211522579193f, -0.10582010447978973f, -0.1608465611934662f, 0.0f, 0.0f, -0.1269841343164444f, -0.21164020895957947f, -0.09312169253826141f, -0.10582010447978973f, 0.0f},
    {0.0f, 0.028218694031238556f, 0.16931216418743134f, 0.033862434327602386f, 0.16931216418743134f, 0.0f, 0.0f, 0.033862434327602386f, 0.16931216418743134f, 0.028218694031238556f, 0.10158730298280716f, 0.0f, 0.0f, 0.022574955597519875f, -0.033862434327602386f, 0.022574955597519875f, -0.05079365149140358f, 0.0f},
    {0.5079365372657776f, 0.6095238327980042f, 0.6095238327980042f, -1.049735426902771f, 2.4719576835632324f, 0.0f, 1.6592592000961304f, 1.0158730745315552f, 1.1174603700637817f, 0.37248677015304565f, 1.8285714387893677f, 0.0f, 0.4740740656852722f, 0.20317460596561432f, 0.10158730298280716f, -0.33862432837486267f, 0.37248677015304565f, 0.0f},
    {0.37248677015304565f, 1.0158730745315552f, 1.8285714387893677f, 1.6592592000961304f, 1.1174603700637817f, 0.0f, -1.049735426902771f, 0.6095238327980042f, 2.4719576835632324f, 0.5079365372657776f, 0.6095238327980042f, 0.0f, -0.33862432837486267f, 0.20317460596561432f, 0.37248677015304565f, 0.4740740656852722f, 0.10158730298280716f, 0.0f},
    {-0.16931216418743134f, -0.33862432837486267f, -0.6095238327980042f, -0.2370370328426361f, -0.7788359522819519f, 0.0f, -0.2370370328426361f, -0.33862432837486267f, -0.7788359522819519f, -0.16931216418743134f, -0.6095238327980042f, 0.0f, -0.20317460596561432f, -0.33862432837486267f, -0.033862434327602386f, -0.20317460596561432f, -0.033862434327602386f, 0.0f},
    {0.31604939699172974f, 0.6320987939834595f, 0.0f, 1.2190476655960083f, 0.0f, 0.0f, 3.566843032836914f, 3.250793695449829f, 0.0f, 2.0317461490631104f, 0.0f, 0.0f, 0.31604939699172974f, 0.31604939699172974f, 0.0f, 0.40634921193122864f, 0.0f, 0.0f},
    {0.06772486865520477f, 0.40634921193122864f, 0.0902998223900795f, 0.0f, 0.5869488716125488f, 0.0f, 0.0902998223900795f, -0.06772486865520477f, 0.0902998223900795f, 0.0f, 0.0f, 0.0f, 0.04514991119503975f, 0.13544973731040955f, 0.022574955597519875f, 0.0f, 0.0902998223900795f, 0.0f},
    {0.028218694031238556f, 0.10158730298280716f, 0.033862434327602386f, 0.0f, 0.16931216418743134f, 0.0f, 0.022574955597519875f, -0.05079365149140358f, 0.022574955597519875f, 0.0f, -0.033862434327602386f, 0.0f, 0.033862434327602386f, 0.16931216418743134f, 0.028218694031238556f, 0.0f, 0.16931216418743134f, 0.0f},
    {0.022574955597519875f, 0.04514991119503975f, 0.04514991119503975f, 0.0f, 0.13544973731040955f, 0.0f, 0.0902998223900795f, 0.06772486865520477f, 0.0902998223900795f, 0.0f, 0.13544973731040955f, 0.0f, 0.0902998223900795f, 0.0902998223900795f, 0.06772486865520477f, 0.0f, 0.13544973731040955f, 0.0f},
    {0.0f, 0.15802469849586487f, 0.31604939699172974f, 0.40634921193122864f, 0.31604939699172974f, 0.0f, 0.0f, 1.6253968477249146f, 3.566843032836914f, 1.0158730745315552f, 1.6253968477249146f, 0.0f, 0.0f, 0.31604939699172974f, 0.31604939699172974f, 0.40634921193122864f, 0.15802469849586487f, 0.0f},
    {0.0f, -0.06208112835884094f, -0.180599644780159f, -0.16931216418743134f, -0.2370370328426361f, 0.0f, 0.0f, -0.42892417311668396f, -1.388359785079956f, -0.3216931223869324f, -0.7788359522819519f, 0.0f, 0.0f, -0.10158730298280716f, 0.04514991119503975f, -0.2370370328426361f, 0.08465608209371567f, 0.0f},
    {0.0f, 0.022574955597519875f, 0.0902998223900795f, 0.04514991119503975f, 0.13544973731040955f, 0.0f, 0.0f, 0.0902998223900795f, 0.5869488716125488f, 0.06772486865520477f, 0.40634921193122864f, 0.0f, 0.0f, 0.0902998223900795f, 0.0f, 0.0902998223900795f, -0.06772486865520477f, 0.0f},
    {0.04514991119503975f, 0.0f, 0.0f, 0.6772486567497253f, -0.40634921193122864f, 0.0f, -0.49664902687072754f, 0.0902998223900795f, -0.49664902687072754f, -0.13544973731040955f, -0.2708994746208191f, 0.0f, -0.0902998223900795f, -0.0902998223900795f, -0.04514991119503975f, 0.2708994746208191f, -0.13544973731040955f, 0.0f},
    {0.22574955224990845f, 0.4514991044998169f, 0.4514991044998169f, -0.40634921193122864f, 1.2190476655960083f, 0.0f, 2.573544979095459f, 2.3477954864501953f, 2.573544979095459f, 0.9481481313705444f, 3.521693229675293f, 0.0f, 0.4514991044998169f, 0.4514991044998169f, 0.22574955224990845f, -0.2708994746208191f, 0.40634921193122864f, 0.0f},
    {-0.04514991119503975f, -0.0902998223900795f, -0.0902998223900795f, 0.13544973731040955f, -0.40634921193122864f, 0.0f, -0.49664902687072754f, -0.4514991044998169f, -0.49664902687072754f, -0.13544973731040955f, -0.8126984238624573f, 0.0f, 0.0f, 0.0f, 0.04514991119503975f, 0.2708994746208191f, -0.13544973731040955f, 0.0f},
    {2.0317461490631104f, 0.0f, 3.250793695449829f, 0.0f, 0.0f, 3.566843032836914f, 0.40634921193122864f, 0.0f, 0.31604939699172974f, 0.0f, 0.0f, 0.31604939699172974f, 1.2190476655960083f, 0.0f, 0.6320987939834595f, 0.0f, 0.0f, 0.31604939699172974f},
    {-0.16931216418743134f, 0.0f, 0.5530864000320435f, 0.0f, 0.0f, -1.388359785079956f, -0.2370370328426361f, 0.0f, 0.022574955597519875f, 0.0f, 0.0f, -0.180599644780159f, -0.9142857193946838f, 0.0f, 0.4740740656852722f, 0.0f, 0.0f, 0.04514991119503975f},
    {0.0f, 0.0f, -0.31604939699172974f, 0.0f, 0.0f, 0.5869488716125488f, 0.0902998223900795f, 0.0f, -0.04514991119503975f, 0.0f, 0.0f, 0.0902998223900795f, 0.5869488716125488f, 0.0f, -0.31604939699172974f, 0.0f, 0.0f, 0.0f},
    {0.0f, 0.13544973731040955f, 0.06772486865520477f, 0.0f, 0.0902998223900795f, 0.0902998223900795f, 0.0f, 0.13544973731040955f, 0.0902998223900795f, 0.0f, 0.06772486865520477f, 0.0902998223900795f, 0.0f, 0.13544973731040955f, 0.04514991119503975f, 0.0f, 0.04514991119503975f, 0.022574955597519875f},
    {0.0f, -0.033862434327602386f, -0.05079365149140358f, 0.0f, 0.022574955597519875f, 0.022574955597519875f, 0.0f, 0.16931216418743134f, 0.16931216418743134f, 0.0f, 0.028218694031238556f, 0.033862434327602386f, 0.0f, 0.16931216418743134f, 0.10158730298280716f, 0.0f, 0.033862434327602386f, 0.028218694031238556f},
    {0.0f, 0.0f, -0.06772486865520477f, 0.0f, 0.0902998223900795f, 0.0902998223900795f, 0.0f, 0.0902998223900795f, 0.13544973731040955f, 0.0f, 0.022574955597519875f, 0.04514991119503975f, 0.0f, 0.5869488716125488f, 0.40634921193122864f, 0.0f, 0.0902998223900795f, 0.06772486865520477f},
    {0.9481481313705444f, 3.521693229675293f, 2.3477954864501953f, 0.0f, 2.573544979095459f, 2.573544979095459f, -0.2708994746208191f, 0.40634921193122864f, 0.4514991044998169f, 0.0f, 0.22574955224990845f, 0.4514991044998169f, -0.40634921193122864f, 1.2190476655960083f, 0.4514991044998169f, 0.0f, 0.4514991044998169f, 0.22574955224990845f},
    {-0.13544973731040955f, -0.8126984238624573f, -0.4514991044998169f, 0.0f, -0.49664902687072754f, -0.49664902687072754f, 0.2708994746208191f, -0.13544973731040955f, 0.0f, 0.0f, 0.04514991119503975f, 0.0f, 0.13544973731040955f, -0.40634921193122864f, -0.0902998223900795f, 0.0f, -0.0902998223900795f, -0.04514991119503975f},
    {-0.13544973731040955f, -0.2708994746208191f, 0.0902998223900795f, 0.0f, -0.49664902687072754f, -0.49664902687072754f, 0.2708994746208191f, -0.13544973731040955f, -0.0902998223900795f, 0.0f, -0.04514991119503975f, -0.0902998223900795f, 0.6772486567497253f, -0.40634921193122864f, 0.0f, 0.0f, 0.0f, 0.04514991119503975f},
    {1.244444489479065f, 0.0f, 1.7777777910232544f, 0.0f, 0.0f, 3.1576719284057617f, 0.49947088956832886f, 0.0f, 0.3301587402820587f, 0.0f, 0.0f, 0.49947088956832886f, 3.1576719284057617f, 0.0f, 1.7777777910232544f, 0.0f, 0.0f, 1.244444489479065f},
    {0.04514991119503975f, 0.0f, 0.4740740656852722f, 0.0f, 0.0f, -0.9142857193946838f, -0.180599644780159f, 0.0f, 0.022574955597519875f, 0.0f, 0.0f, -0.2370370328426361f, -1.388359785079956f, 0.0f, 0.5530864000320435f, 0.0f, 0.0f, -0.16931216418743134f},
    {0.0f, 0.16931216418743134f, 0.028218694031238556f, 0.0f, 0.16931216418743134f, 0.033862434327602386f, 0.0f, -0.033862434327602386f, 0.022574955597519875f, 0.0f, -0.05079365149140358f, 0.022574955597519875f, 0.0f, 0.16931216418743134f, 0.033862434327602386f, 0.0f, 0.10158730298280716f, 0.028218694031238556f},
    {0.0f, -0.21164020895957947f, -0.10582010447978973f, 0.0f, -0.1269841343164444f, -0.09312169253826141f, 0.0f, -0.21164020895957947f, -0.1269841343164444f, 0.0f, -0.10582010447978973f, -0.09312169253826141f, 0.0f, -0.3640211522579193f, -0.1608465611934662f, 0.0f, -0.1608465611934662f, -0.10582010447978973f},
    {0.0f, 0.04514991119503975f, 0.08465608209371567f, 0.0f, -0.10158730298280716f, -0.2370370328426361f, 0.0f, -0.180599644780159f, -0.2370370328426361f, 0.0f, -0.06208112835884094f, -0.16931216418743134f, 0.0f, -1.388359785079956f, -0.7788359522819519f, 0.0f, -0.42892417311668396f, -0.3216931223869324f},
    {0.5079365372657776f, 0.6095238327980042f, 0.6095238327980042f, 0.0f, 2.4719576835632324f, -1.049735426902771f, 0.4740740656852722f, 0.10158730298280716f, 0.20317460596561432f, 0.0f, 0.37248677015304565f, -0.33862432837486267f, 1.6592592000961304f, 1.1174603700637817f, 1.0158730745315552f, 0.0f, 1.8285714387893677f, 0.37248677015304565f},
    {-0.16931216418743134f, -0.6095238327980042f, -0.33862432837486267f, 0.0f, -0.7788359522819519f, -0.2370370328426361f, -0.20317460596561432f, -0.033862434327602386f, -0.33862432837486267f, 0.0f, -0.033862434327602386f, -0.20317460596561432f, -0.2370370328426361f, -0.7788359522819519f, -0.33862432837486267f, 0.0f, -0.6095238327980042f, -0.16931216418743134f},
    {0.37248677015304565f, 1.8285714387893677f, 1.0158730745315552f, 0.0f, 1.1174603700637817f, 1.6592592000961304f, -0.33862432837486267f, 0.37248677015304565f, 0.20317460596561432f, 0.0f, 0.10158730298280716f, 0.4740740656852722f, -1.049735426902771f, 2.4719576835632324f, 0.6095238327980042f, 0.0f, 0.6095238327980042f, 0.5079365372657776f},
    {0.31604939699172974f, 0.0f, 0.6320987939834595f, 0.0f, 0.0f, 1.2190476655960083f, 0.31604939699172974f, 0.0f, 0.31604939699172974f, 0.0f, 0.0f, 0.40634921193122864f, 3.566843032836914f, 0.0f, 3.250793695449829f, 0.0f, 0.0f, 2.0317461490631104f},
    {0.0f, 0.0902998223900795f, 0.022574955597519875f, 0.0f, 0.13544973731040955f, 0.04514991119503975f, 0.0f, 0.0f, 0.0902998223900795f, 0.0f, -0.06772486865520477f, 0.0902998223900795f, 0.0f, 0.5869488716125488f, 0.0902998223900795f, 0.0f, 0.40634921193122864f, 0.06772486865520477f},
    {0.0f, -0.180599644780159f, -0.06208112835884094f, 0.0f, -0.2370370328426361f, -0.16931216418743134f, 0.0f, 0.04514991119503975f, -0.10158730298280716f, 0.0f, 0.08465608209371567f, -0.2370370328426361f, 0.0f, -1.388359785079956f, -0.42892417311668396f, 0.0f, -0.7788359522819519f, -0.3216931223869324f},
    {0.0f, 0.31604939699172974f, 0.15802469849586487f, 0.0f, 0.31604939699172974f, 0.40634921193122864f, 0.0f, 0.31604939699172974f, 0.31604939699172974f, 0.0f, 0.15802469849586487f, 0.40634921193122864f, 0.0f, 3.566843032836914f, 1.6253968477249146f, 0.0f, 1.6253968477249146f, 1.0158730745315552f},
    {0.04514991119503975f, 0.0f, 0.0f, 0.0f, -0.40634921193122864f, 0.6772486567497253f, -0.0902998223900795f, -0.04514991119503975f, -0.0902998223900795f, 0.0f, -0.13544973731040955f, 0.2708994746208191f, -0.49664902687072754f, -0.49664902687072754f, 0.0902998223900795f, 0.0f, -0.2708994746208191f, -0.13544973731040955f},
    {-0.04514991119503975f, -0.0902998223900795f, -0.0902998223900795f, 0.0f, -0.40634921193122864f, 0.13544973731040955f, 0.0f, 0.04514991119503975f, 0.0f, 0.0f, -0.13544973731040955f, 0.2708994746208191f, -0.49664902687072754f, -0.49664902687072754f, -0.4514991044998169f, 0.0f, -0.8126984238624573f, -0.13544973731040955f},
    {0.22574955224990845f, 0.4514991044998169f, 0.4514991044998169f, 0.0f, 1.2190476655960083f, -0.40634921193122864f, 0.4514991044998169f, 0.22574955224990845f, 0.4514991044998169f, 0.0f, 0.40634921193122864f, -0.2708994746208191f, 2.573544979095459f, 2.573544979095459f, 2.3477954864501953f, 0.0f, 3.521693229675293f, 0.9481481313705444f},
    {0.0f, 0.0f, 0.0f, 0.40634921193122864f, 0.31604939699172974f, 0.31604939699172974f, 0.0f, 0.0f, 0.0f, 2.0317461490631104f, 3.250793695449829f, 3.566843032836914f, 0.0f, 0.0f, 0.0f, 1.2190476655960083f, 0.6320987939834595f, 0.31604939699172974f},
    {0.0f, 0.0f, 0.0f, -0.2370370328426361f, 0.022574955597519875f, -0.180599644780159f, 0.0f, 0.0f, 0.0f, -0.16931216418743134f, 0.5530864000320435f, -1.388359785079956f, 0.0f, 0.0f, 0.0f, -0.9142857193946838f, 0.4740740656852722f, 0.04514991119503975f},
    {0.0f, 0.0f, 0.0f, 0.0902998223900795f, -0.04514991119503975f, 0.0902998223900795f, 0.0f, 0.0f, 0.0f, 0.0f, -0.31604939699172974f, 0.5869488716125488f, 0.0f, 0.0f, 0.0f, 0.5869488716125488f, -0.31604939699172974f, 0.0f},
    {0.0f, -0.13544973731040955f, 0.04514991119503975f, 0.2708994746208191f, 0.0f, 0.0f, 0.0f, -0.8126984238624573f, -0.49664902687072754f, -0.13544973731040955f, -0.4514991044998169f, -0.49664902687072754f, 0.0f, -0.40634921193122864f, -0.0902998223900795f, 0.13544973731040955f, -0.0902998223900795f, -0.04514991119503975f},
    {0.0f, 0.40634921193122864f, 0.22574955224990845f, -0.2708994746208191f, 0.4514991044998169f, 0.4514991044998169f, 0.0f, 3.521693229675293f, 2.573544979095459f, 0.9481481313705444f, 2.3477954864501953f, 2.573544979095459f, 0.0f, 1.2190476655960083f, 0.4514991044998169f, -0.40634921193122864f, 0.4514991044998169f, 0.22574955224990845f},
    {0.0f, -0.13544973731040955f, -0.04514991119503975f, 0.2708994746208191f, -0.0902998223900795f, -0.0902998223900795f, 0.0f, -0.2708994746208191f, -0.49664902687072754f, -0.13544973731040955f, 0.0902998223900795f, -0.49664902687072754f, 0.0f, -0.40634921193122864f, 0.0f, 0.6772486567497253f, 0.0f, 0.04514991119503975f},
    {0.0f, 0.0f, 0.0f, 0.49947088956832886f, 0.3301587402820587f, 0.49947088956832886f, 0.0f, 0.0f, 0.0f, 1.244444489479065f, 1.7777777910232544f, 3.1576719284057617f, 0.0f, 0.0f, 0.0f, 3.1576719284057617f, 1.7777777910232544f, 1.244444489479065f},
    {0.0f, 0.0f, 0.0f, -0.180599644780159f, 0.022574955597519875f, -0.2370370328426361f, 0.0f, 0.0f, 0.0f, 0.04514991119503975f, 0.4740740656852722f, -0.9142857193946838f, 0.0f, 0.0f, 0.0f, -1.388359785079956f, 0.5530864000320435f, -0.16931216418743134f},
    {0.0f, -0.033862434327602386f, -0.033862434327602386f, -0.20317460596561432f, -0.33862432837486267f, -0.20317460596561432f, 0.0f, -0.6095238327980042f, -0.7788359522819519f, -0.16931216418743134f, -0.33862432837486267f, -0.2370370328426361f, 0.0f, -0.7788359522819519f, -0.6095238327980042f, -0.2370370328426361f, -0.33862432837486267f, -0.16931216418743134f},
    {0.0f, 0.10158730298280716f, 0.37248677015304565f, 0.4740740656852722f, 0.20317460596561432f, -0.33862432837486267f, 0.0f, 0.6095238327980042f, 2.4719576835632324f, 0.5079365372657776f, 0.6095238327980042f, -1.049735426902771f, 0.0f, 1.1174603700637817f, 1.8285714387893677f, 1.6592592000961304f, 1.0158730745315552f, 0.37248677015304565f},
    {0.0f, 0.37248677015304565f, 0.10158730298280716f, -0.33862432837486267f, 0.20317460596561432f, 0.4740740656852722f, 0.0f, 1.8285714387893677f, 1.1174603700637817f, 0.37248677015304565f, 1.0158730745315552f, 1.6592592000961304f, 0.0f, 2.4719576835632324f, 0.6095238327980042f, -1.049735426902771f, 0.6095238327980042f, 0.5079365372657776f},
    {0.0f, 0.0f, 0.0f, 0.31604939699172974f, 0.31604939699172974f, 0.40634921193122864f, 0.0f, 0.0f, 0.0f, 0.31604939699172974f, 0.6320987939834595f, 1.2190476655960083f, 0.0f, 0.0f, 0.0f, 3.566843032836914f, 3.250793695449829f, 2.0317461490631104f},
    {0.0f, 0.04514991119503975f, -0.13544973731040955f, 0.0f, 0.0f, 0.2708994746208191f, 0.0f, -0.0902998223900795f, -0.40634921193122864f, -0.04514991119503975f, -0.0902998223900795f, 0.13544973731040955f, 0.0f, -0.49664902687072754f, -0.8126984238624573f, -0.49664902687072754f, -0.4514991044998169f, -0.13544973731040955f},
    {0.0f, -0.04514991119503975f, -0.13544973731040955f, -0.0902998223900795f, -0.0902998223900795f, 0.2708994746208191f, 0.0f, 0.0f, -0.40634921193122864f, 0.04514991119503975f, 0.0f, 0.6772486567497253f, 0.0f, -0.49664902687072754f, -0.2708994746208191f, -0.49664902687072754f, 0.0902998223900795f, -0.13544973731040955f},
    {0.0f, 0.22574955224990845f, 0.40634921193122864f, 0.4514991044998169f, 0.4514991044998169f, -0.2708994746208191f, 0.0f, 0.4514991044998169f, 1.2190476655960083f, 0.22574955224990845f, 0.4514991044998169f, -0.40634921193122864f, 0.0f, 2.573544979095459f, 3.521693229675293f, 2.573544979095459f, 2.3477954864501953f, 0.9481481313705444f},
    {3.7925925254821777f, 5.9597883224487305f, 5.9597883224487305f, 7.043386459350586f, 7.043386459350586f, 7.043386459350586f, 3.7925925254821777f, 2.1671957969665527f, 3.250793695449829f, 1.0835978984832764f, 2.1671957969665527f, 3.250793695449829f, 3.7925925254821777f, 3.250793695449829f, 2.1671957969665527f, 3.250793695449829f, 2.1671957969665527f, 1.0835978984832764f},
    {0.2708994746208191f, 1.8962962627410889f, 0.8126984238624573f, -1.0835978984832764f, 0.8126984238624573f, 0.8126984238624573f, -1.0835978984832764f, 1.8962962627410889f, 0.8126984238624573f, 0.2708994746208191f, 0.8126984238624573f, 0.8126984238624573f, -0.8126984238624573f, 1.0835978984832764f, 0.0f, -0.8126984238624573f, 0.0f, 0.0f},
    {0.2708994746208191f, 0.8126984238624573f, 1.8962962627410889f, 0.8126984238624573f, 0.8126984238624573f, -1.0835978984832764f, -0.8126984238624573f, 0.0f, 1.0835978984832764f, 0.0f, 0.0f, -0.8126984238624573f, -1.0835978984832764f, 0.8126984238624573f, 1.8962962627410889f, 0.8126984238624573f, 0.8126984238624573f, 0.2708994746208191f},
    {1.0835978984832764f, 2.1671957969665527f, 2.1671957969665527f, 3.7925925254821777f, 3.250793695449829f, 3.250793695449829f, 7.043386459350586f, 5.9597883224487305f, 7.043386459350586f, 3.7925925254821777f, 5.9597883224487305f, 7.043386459350586f, 3.250793695449829f, 3.250793695449829f, 2.1671957969665527f, 3.7925925254821777f, 2.1671957969665527f, 1.0835978984832764f},
    {0.0f, 0.0f, 0.0f, -0.8126984238624573f, 1.0835978984832764f, -0.8126984238624573f, 0.8126984238624573f, 0.8126984238624573f, 0.8126984238624573f, 0.2708994746208191f, 1.8962962627410889f, -1.0835978984832764f, 0.8126984238624573f, 0.8126984238624573f, 0.8126984238624573f, -1.0835978984832764f, 1.8962962627410889f, 0.2708994746208191f},
    {1.0835978984832764f, 2.1671957969665527f, 2.1671957969665527f, 3.250793695449829f, 3.250793695449829f, 3.7925925254821777f, 3.250793695449829f, 2.1671957969665527f, 3.250793695449829f, 1.0835978984832764f, 2.1671957969665527f, 3.7925925254821777f, 7.043386459350586f, 7.043386459350586f, 5.9597883224487305f, 7.043386459350586f, 5.9597883224487305f, 3.7925925254821777f}};
#endif

}  // namespace fe_gen
