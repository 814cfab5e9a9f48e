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
  template <class Ops> __device__ __forceinline__ static void stiffness_upper(const typename Ops::T* Lam, typename Ops::T* K) {
    K[0] = Lam[0];
    K[1] = Lam[1];
    K[2] = Lam[2];
    K[3] = Lam[3];
    K[4] = Lam[4];
    K[5] = Lam[5];
  }
  template <class Ops> __device__ __forceinline__ static void mass_upper_add(const typename Ops::T& vol, typename Ops::T* K) {
    K[0] = Ops::fmac(vol, 0.16666666666666666, K[0]);
    K[1] = Ops::fmac(vol, 0.08333333333333333, K[1]);
    K[2] = Ops::fmac(vol, 0.08333333333333333, K[2]);
    K[3] = Ops::fmac(vol, 0.16666666666666666, K[3]);
    K[4] = Ops::fmac(vol, 0.08333333333333333, K[4]);
    K[5] = Ops::fmac(vol, 0.16666666666666666, K[5]);
  }
  template <class Ops> __device__ __forceinline__ static void mass_upper(const typename Ops::T& vol, typename Ops::T* K) {
    K[0] = Ops::mulc(vol, 0.16666666666666666);
    K[1] = Ops::mulc(vol, 0.08333333333333333);
    K[2] = Ops::mulc(vol, 0.08333333333333333);
    K[3] = Ops::mulc(vol, 0.16666666666666666);
    K[4] = Ops::mulc(vol, 0.08333333333333333);
    K[5] = Ops::mulc(vol, 0.16666666666666666);
  }
  template <class Ops, bool STIFF, bool MASS> __device__ __forceinline__ static void action_upper(const typename Ops::T* Lam, const typename Ops::T& vol, const typename Ops::T* x, typename Ops::T* y) {
    typename Ops::T k;
    { if constexpr (STIFF) { k = Lam[0]; } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, 0.16666666666666666, k); } y[0] = Ops::fma3(k, x[0], y[0]); }
    { if constexpr (STIFF) { k = Lam[1]; } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, 0.08333333333333333, k); } y[0] = Ops::fma3(k, x[1], y[0]); y[1] = Ops::fma3(k, x[0], y[1]); }
    { if constexpr (STIFF) { k = Lam[2]; } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, 0.08333333333333333, k); } y[0] = Ops::fma3(k, x[2], y[0]); y[2] = Ops::fma3(k, x[0], y[2]); }
    { if constexpr (STIFF) { k = Lam[3]; } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, 0.16666666666666666, k); } y[1] = Ops::fma3(k, x[1], y[1]); }
    { if constexpr (STIFF) { k = Lam[4]; } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, 0.08333333333333333, k); } y[1] = Ops::fma3(k, x[2], y[1]); y[2] = Ops::fma3(k, x[1], y[2]); }
    { if constexpr (STIFF) { k = Lam[5]; } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, 0.16666666666666666, k); } y[2] = Ops::fma3(k, x[2], y[2]); }
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
  template <class Ops> __device__ __forceinline__ static void stiffness_upper(const typename Ops::T* Lam, typename Ops::T* K) {
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
    K[15] = Ops::fmac(Lam[3], 2.6666666666666665, Ops::fmac(Lam[1], 2.6666666666666665, Ops::mulc(Lam[0], 2.6666666666666665)));
    K[16] = Ops::fmac(Lam[4], 2.6666666666666665, Ops::fmac(Lam[2], 1.3333333333333333, Ops::fmac(Lam[1], 1.3333333333333333, Ops::mulc(Lam[0], 1.3333333333333333))));
    K[17] = Ops::fmac(Lam[4], 1.3333333333333333, Ops::fmac(Lam[3], 1.3333333333333333, Ops::fmac(Lam[2], 2.6666666666666665, Ops::mulc(Lam[1], 1.3333333333333333))));
    K[18] = Ops::fmac(Lam[5], 2.6666666666666665, Ops::fmac(Lam[2], 2.6666666666666665, Ops::mulc(Lam[0], 2.6666666666666665)));
    K[19] = Ops::fmac(Lam[5], 1.3333333333333333, Ops::fmac(Lam[4], 1.3333333333333333, Ops::fmac(Lam[2], 1.3333333333333333, Ops::mulc(Lam[1], 2.6666666666666665))));
    K[20] = Ops::fmac(Lam[5], 2.6666666666666665, Ops::fmac(Lam[4], 2.6666666666666665, Ops::mulc(Lam[3], 2.6666666666666665)));
  }
  template <class Ops> __device__ __forceinline__ static void mass_upper_add(const typename Ops::T& vol, typename Ops::T* K) {
    K[0] = Ops::fmac(vol, 0.03333333333333333, K[0]);
    K[1] = Ops::fmac(vol, -0.005555555555555556, K[1]);
    K[2] = Ops::fmac(vol, -0.005555555555555556, K[2]);
    K[5] = Ops::fmac(vol, -0.022222222222222223, K[5]);
    K[6] = Ops::fmac(vol, 0.03333333333333333, K[6]);
    K[7] = Ops::fmac(vol, -0.005555555555555556, K[7]);
    K[9] = Ops::fmac(vol, -0.022222222222222223, K[9]);
    K[11] = Ops::fmac(vol, 0.03333333333333333, K[11]);
    K[12] = Ops::fmac(vol, -0.022222222222222223, K[12]);
    K[15] = Ops::fmac(vol, 0.17777777777777778, K[15]);
    K[16] = Ops::fmac(vol, 0.08888888888888889, K[16]);
    K[17] = Ops::fmac(vol, 0.08888888888888889, K[17]);
    K[18] = Ops::fmac(vol, 0.17777777777777778, K[18]);
    K[19] = Ops::fmac(vol, 0.08888888888888889, K[19]);
    K[20] = Ops::fmac(vol, 0.17777777777777778, K[20]);
  }
  template <class Ops> __device__ __forceinline__ static void mass_upper(const typename Ops::T& vol, typename Ops::T* K) {
    K[0] = Ops::mulc(vol, 0.03333333333333333);
    K[1] = Ops::mulc(vol, -0.005555555555555556);
    K[2] = Ops::mulc(vol, -0.005555555555555556);
    K[3] = Ops::mulc(vol, 0.0);
    K[4] = Ops::mulc(vol, 0.0);
    K[5] = Ops::mulc(vol, -0.022222222222222223);
    K[6] = Ops::mulc(vol, 0.03333333333333333);
    K[7] = Ops::mulc(vol, -0.005555555555555556);
    K[8] = Ops::mulc(vol, 0.0);
    K[9] = Ops::mulc(vol, -0.022222222222222223);
    K[10] = Ops::mulc(vol, 0.0);
    K[11] = Ops::mulc(vol, 0.03333333333333333);
    K[12] = Ops::mulc(vol, -0.022222222222222223);
    K[13] = Ops::mulc(vol, 0.0);
    K[14] = Ops::mulc(vol, 0.0);
    K[15] = Ops::mulc(vol, 0.17777777777777778);
    K[16] = Ops::mulc(vol, 0.08888888888888889);
    K[17] = Ops::mulc(vol, 0.08888888888888889);
    K[18] = Ops::mulc(vol, 0.17777777777777778);
    K[19] = Ops::mulc(vol, 0.08888888888888889);
    K[20] = Ops::mulc(vol, 0.17777777777777778);
  }
  template <class Ops, bool STIFF, bool MASS> __device__ __forceinline__ static void action_upper(const typename Ops::T* Lam, const typename Ops::T& vol, const typename Ops::T* x, typename Ops::T* y) {
    typename Ops::T k;
    { if constexpr (STIFF) { k = Lam[0]; } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, 0.03333333333333333, k); } y[0] = Ops::fma3(k, x[0], y[0]); }
    { if constexpr (STIFF) { k = Ops::mulc(Lam[1], -0.3333333333333333); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, -0.005555555555555556, k); } y[0] = Ops::fma3(k, x[1], y[0]); y[1] = Ops::fma3(k, x[0], y[1]); }
    { if constexpr (STIFF) { k = Ops::mulc(Lam[2], -0.3333333333333333); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, -0.005555555555555556, k); } y[0] = Ops::fma3(k, x[2], y[0]); y[2] = Ops::fma3(k, x[0], y[2]); }
    if constexpr (STIFF) { if constexpr (STIFF) { k = Ops::mulc(Lam[1], 1.3333333333333333); } else { k = Ops::zero(); } y[0] = Ops::fma3(k, x[3], y[0]); y[3] = Ops::fma3(k, x[0], y[3]); }
    if constexpr (STIFF) { if constexpr (STIFF) { k = Ops::mulc(Lam[2], 1.3333333333333333); } else { k = Ops::zero(); } y[0] = Ops::fma3(k, x[4], y[0]); y[4] = Ops::fma3(k, x[0], y[4]); }
    if constexpr (MASS) { k = Ops::zero(); if constexpr (MASS) { k = Ops::fmac(vol, -0.022222222222222223, k); } y[0] = Ops::fma3(k, x[5], y[0]); y[5] = Ops::fma3(k, x[0], y[5]); }
    { if constexpr (STIFF) { k = Lam[3]; } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, 0.03333333333333333, k); } y[1] = Ops::fma3(k, x[1], y[1]); }
    { if constexpr (STIFF) { k = Ops::mulc(Lam[4], -0.3333333333333333); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, -0.005555555555555556, k); } y[1] = Ops::fma3(k, x[2], y[1]); y[2] = Ops::fma3(k, x[1], y[2]); }
    if constexpr (STIFF) { if constexpr (STIFF) { k = Ops::mulc(Lam[1], 1.3333333333333333); } else { k = Ops::zero(); } y[1] = Ops::fma3(k, x[3], y[1]); y[3] = Ops::fma3(k, x[1], y[3]); }
    if constexpr (MASS) { k = Ops::zero(); if constexpr (MASS) { k = Ops::fmac(vol, -0.022222222222222223, k); } y[1] = Ops::fma3(k, x[4], y[1]); y[4] = Ops::fma3(k, x[1], y[4]); }
    if constexpr (STIFF) { if constexpr (STIFF) { k = Ops::mulc(Lam[4], 1.3333333333333333); } else { k = Ops::zero(); } y[1] = Ops::fma3(k, x[5], y[1]); y[5] = Ops::fma3(k, x[1], y[5]); }
    { if constexpr (STIFF) { k = Lam[5]; } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, 0.03333333333333333, k); } y[2] = Ops::fma3(k, x[2], y[2]); }
    if constexpr (MASS) { k = Ops::zero(); if constexpr (MASS) { k = Ops::fmac(vol, -0.022222222222222223, k); } y[2] = Ops::fma3(k, x[3], y[2]); y[3] = Ops::fma3(k, x[2], y[3]); }
    if constexpr (STIFF) { if constexpr (STIFF) { k = Ops::mulc(Lam[2], 1.3333333333333333); } else { k = Ops::zero(); } y[2] = Ops::fma3(k, x[4], y[2]); y[4] = Ops::fma3(k, x[2], y[4]); }
    if constexpr (STIFF) { if constexpr (STIFF) { k = Ops::mulc(Lam[4], 1.3333333333333333); } else { k = Ops::zero(); } y[2] = Ops::fma3(k, x[5], y[2]); y[5] = Ops::fma3(k, x[2], y[5]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[3], 2.6666666666666665, Ops::fmac(Lam[1], 2.6666666666666665, Ops::mulc(Lam[0], 2.6666666666666665))); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, 0.17777777777777778, k); } y[3] = Ops::fma3(k, x[3], y[3]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[4], 2.6666666666666665, Ops::fmac(Lam[2], 1.3333333333333333, Ops::fmac(Lam[1], 1.3333333333333333, Ops::mulc(Lam[0], 1.3333333333333333)))); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, 0.08888888888888889, k); } y[3] = Ops::fma3(k, x[4], y[3]); y[4] = Ops::fma3(k, x[3], y[4]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[4], 1.3333333333333333, Ops::fmac(Lam[3], 1.3333333333333333, Ops::fmac(Lam[2], 2.6666666666666665, Ops::mulc(Lam[1], 1.3333333333333333)))); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, 0.08888888888888889, k); } y[3] = Ops::fma3(k, x[5], y[3]); y[5] = Ops::fma3(k, x[3], y[5]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[5], 2.6666666666666665, Ops::fmac(Lam[2], 2.6666666666666665, Ops::mulc(Lam[0], 2.6666666666666665))); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, 0.17777777777777778, k); } y[4] = Ops::fma3(k, x[4], y[4]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[5], 1.3333333333333333, Ops::fmac(Lam[4], 1.3333333333333333, Ops::fmac(Lam[2], 1.3333333333333333, Ops::mulc(Lam[1], 2.6666666666666665)))); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, 0.08888888888888889, k); } y[4] = Ops::fma3(k, x[5], y[4]); y[5] = Ops::fma3(k, x[4], y[5]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[5], 2.6666666666666665, Ops::fmac(Lam[4], 2.6666666666666665, Ops::mulc(Lam[3], 2.6666666666666665))); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, 0.17777777777777778, k); } y[5] = Ops::fma3(k, x[5], y[5]); }
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
  template <class Ops> __device__ __forceinline__ static void stiffness_upper(const typename Ops::T* Lam, typename Ops::T* K) {
    K[0] = Ops::mulc(Lam[0], 0.85);
    K[1] = Ops::mulc(Lam[1], 0.175);
    K[2] = Ops::mulc(Lam[2], 0.175);
    K[3] = Ops::fmac(Lam[1], 1.425, Ops::mulc(Lam[0], 0.075));
    K[4] = Ops::fmac(Lam[1], -0.6, Ops::mulc(Lam[0], 0.075));
    K[5] = Ops::fmac(Lam[2], 1.425, Ops::mulc(Lam[0], 0.075));
    K[6] = Ops::fmac(Lam[2], -0.6, Ops::mulc(Lam[0], 0.075));
    K[7] = Ops::fmac(Lam[2], 0.075, Ops::mulc(Lam[1], 0.075));
    K[8] = Ops::fmac(Lam[2], 0.075, Ops::mulc(Lam[1], 0.075));
    K[9] = Ops::fmac(Lam[2], 0.225, Ops::fmac(Lam[1], 0.225, Ops::mulc(Lam[0], 0.225)));
    K[10] = Ops::mulc(Lam[3], 0.85);
    K[11] = Ops::mulc(Lam[4], 0.175);
    K[12] = Ops::fmac(Lam[3], 0.075, Ops::mulc(Lam[1], -0.6));
    K[13] = Ops::fmac(Lam[3], 0.075, Ops::mulc(Lam[1], 1.425));
    K[14] = Ops::fmac(Lam[4], 0.075, Ops::mulc(Lam[1], 0.075));
    K[15] = Ops::fmac(Lam[4], 0.075, Ops::mulc(Lam[1], 0.075));
    K[16] = Ops::fmac(Lam[4], 1.425, Ops::mulc(Lam[3], 0.075));
    K[17] = Ops::fmac(Lam[4], -0.6, Ops::mulc(Lam[3], 0.075));
    K[18] = Ops::fmac(Lam[4], 0.225, Ops::fmac(Lam[3], 0.225, Ops::mulc(Lam[1], 0.225)));
    K[19] = Ops::mulc(Lam[5], 0.85);
    K[20] = Ops::fmac(Lam[4], 0.075, Ops::mulc(Lam[2], 0.075));
    K[21] = Ops::fmac(Lam[4], 0.075, Ops::mulc(Lam[2], 0.075));
    K[22] = Ops::fmac(Lam[5], 0.075, Ops::mulc(Lam[2], -0.6));
    K[23] = Ops::fmac(Lam[5], 0.075, Ops::mulc(Lam[2], 1.425));
    K[24] = Ops::fmac(Lam[5], 0.075, Ops::mulc(Lam[4], -0.6));
    K[25] = Ops::fmac(Lam[5], 0.075, Ops::mulc(Lam[4], 1.425));
    K[26] = Ops::fmac(Lam[5], 0.225, Ops::fmac(Lam[4], 0.225, Ops::mulc(Lam[2], 0.225)));
    K[27] = Ops::fmac(Lam[3], 3.375, Ops::fmac(Lam[1], 3.375, Ops::mulc(Lam[0], 3.375)));
    K[28] = Ops::fmac(Lam[3], -0.675, Ops::fmac(Lam[1], 1.35, Ops::mulc(Lam[0], -0.675)));
    K[29] = Ops::fmac(Lam[4], 3.375, Ops::fmac(Lam[2], 1.6875, Ops::fmac(Lam[1], 1.6875, Ops::mulc(Lam[0], 1.6875))));
    K[30] = Ops::fmac(Lam[4], -0.675, Ops::fmac(Lam[2], -0.3375, Ops::fmac(Lam[1], -0.3375, Ops::mulc(Lam[0], -0.3375))));
    K[31] = Ops::fmac(Lam[4], -0.3375, Ops::fmac(Lam[3], -0.3375, Ops::fmac(Lam[2], -0.675, Ops::mulc(Lam[1], -0.3375))));
    K[32] = Ops::fmac(Lam[4], -0.3375, Ops::fmac(Lam[3], -0.3375, Ops::fmac(Lam[2], -0.675, Ops::mulc(Lam[1], -0.3375))));
    K[33] = Ops::fmac(Lam[4], 2.025, Ops::fmac(Lam[3], 2.025, Ops::fmac(Lam[2], 4.05, Ops::mulc(Lam[1], 2.025))));
    K[34] = Ops::fmac(Lam[3], 3.375, Ops::fmac(Lam[1], 3.375, Ops::mulc(Lam[0], 3.375)));
    K[35] = Ops::fmac(Lam[4], -0.675, Ops::fmac(Lam[2], -0.3375, Ops::fmac(Lam[1], -0.3375, Ops::mulc(Lam[0], -0.3375))));
    K[36] = Ops::fmac(Lam[4], -0.675, Ops::fmac(Lam[2], -0.3375, Ops::fmac(Lam[1], -0.3375, Ops::mulc(Lam[0], -0.3375))));
    K[37] = Ops::fmac(Lam[4], 1.6875, Ops::fmac(Lam[3], 1.6875, Ops::fmac(Lam[2], 3.375, Ops::mulc(Lam[1], 1.6875))));
    K[38] = Ops::fmac(Lam[4], -0.3375, Ops::fmac(Lam[3], -0.3375, Ops::fmac(Lam[2], -0.675, Ops::mulc(Lam[1], -0.3375))));
    K[39] = Ops::fmac(Lam[4], 4.05, Ops::fmac(Lam[2], 2.025, Ops::fmac(Lam[1], 2.025, Ops::mulc(Lam[0], 2.025))));
    K[40] = Ops::fmac(Lam[5], 3.375, Ops::fmac(Lam[2], 3.375, Ops::mulc(Lam[0], 3.375)));
    K[41] = Ops::fmac(Lam[5], -0.675, Ops::fmac(Lam[2], 1.35, Ops::mulc(Lam[0], -0.675)));
    K[42] = Ops::fmac(Lam[5], -0.3375, Ops::fmac(Lam[4], -0.3375, Ops::fmac(Lam[2], -0.3375, Ops::mulc(Lam[1], -0.675))));
    K[43] = Ops::fmac(Lam[5], -0.3375, Ops::fmac(Lam[4], -0.3375, Ops::fmac(Lam[2], -0.3375, Ops::mulc(Lam[1], -0.675))));
    K[44] = Ops::fmac(Lam[5], 2.025, Ops::fmac(Lam[4], 2.025, Ops::fmac(Lam[2], 2.025, Ops::mulc(Lam[1], 4.05))));
    K[45] = Ops::fmac(Lam[5], 3.375, Ops::fmac(Lam[2], 3.375, Ops::mulc(Lam[0], 3.375)));
    K[46] = Ops::fmac(Lam[5], -0.3375, Ops::fmac(Lam[4], -0.3375, Ops::fmac(Lam[2], -0.3375, Ops::mulc(Lam[1], -0.675))));
    K[47] = Ops::fmac(Lam[5], 1.6875, Ops::fmac(Lam[4], 1.6875, Ops::fmac(Lam[2], 1.6875, Ops::mulc(Lam[1], 3.375))));
    K[48] = Ops::fmac(Lam[4], 4.05, Ops::fmac(Lam[2], 2.025, Ops::fmac(Lam[1], 2.025, Ops::mulc(Lam[0], 2.025))));
    K[49] = Ops::fmac(Lam[5], 3.375, Ops::fmac(Lam[4], 3.375, Ops::mulc(Lam[3], 3.375)));
    K[50] = Ops::fmac(Lam[5], -0.675, Ops::fmac(Lam[4], 1.35, Ops::mulc(Lam[3], -0.675)));
    K[51] = Ops::fmac(Lam[5], 2.025, Ops::fmac(Lam[4], 2.025, Ops::fmac(Lam[2], 2.025, Ops::mulc(Lam[1], 4.05))));
    K[52] = Ops::fmac(Lam[5], 3.375, Ops::fmac(Lam[4], 3.375, Ops::mulc(Lam[3], 3.375)));
    K[53] = Ops::fmac(Lam[4], 2.025, Ops::fmac(Lam[3], 2.025, Ops::fmac(Lam[2], 4.05, Ops::mulc(Lam[1], 2.025))));
    K[54] = Ops::fmac(Lam[5], 8.1, Ops::fmac(Lam[4], 8.1, Ops::fmac(Lam[3], 8.1, Ops::fmac(Lam[2], 8.1, Ops::fmac(Lam[1], 8.1, Ops::mulc(Lam[0], 8.1))))));
  }
  template <class Ops> __device__ __forceinline__ static void mass_upper_add(const typename Ops::T& vol, typename Ops::T* K) {
    K[0] = Ops::fmac(vol, 0.01130952380952381, K[0]);
    K[1] = Ops::fmac(vol, 0.001636904761904762, K[1]);
    K[2] = Ops::fmac(vol, 0.001636904761904762, K[2]);
    K[3] = Ops::fmac(vol, 0.0026785714285714286, K[3]);
    K[5] = Ops::fmac(vol, 0.0026785714285714286, K[5]);
    K[7] = Ops::fmac(vol, 0.0040178571428571425, K[7]);
    K[8] = Ops::fmac(vol, 0.0040178571428571425, K[8]);
    K[9] = Ops::fmac(vol, 0.005357142857142857, K[9]);
    K[10] = Ops::fmac(vol, 0.01130952380952381, K[10]);
    K[11] = Ops::fmac(vol, 0.001636904761904762, K[11]);
    K[13] = Ops::fmac(vol, 0.0026785714285714286, K[13]);
    K[14] = Ops::fmac(vol, 0.0040178571428571425, K[14]);
    K[15] = Ops::fmac(vol, 0.0040178571428571425, K[15]);
    K[16] = Ops::fmac(vol, 0.0026785714285714286, K[16]);
    K[18] = Ops::fmac(vol, 0.005357142857142857, K[18]);
    K[19] = Ops::fmac(vol, 0.01130952380952381, K[19]);
    K[20] = Ops::fmac(vol, 0.0040178571428571425, K[20]);
    K[21] = Ops::fmac(vol, 0.0040178571428571425, K[21]);
    K[23] = Ops::fmac(vol, 0.0026785714285714286, K[23]);
    K[25] = Ops::fmac(vol, 0.0026785714285714286, K[25]);
    K[26] = Ops::fmac(vol, 0.005357142857142857, K[26]);
    K[27] = Ops::fmac(vol, 0.08035714285714286, K[27]);
    K[28] = Ops::fmac(vol, -0.028125, K[28]);
    K[29] = Ops::fmac(vol, 0.04017857142857143, K[29]);
    K[30] = Ops::fmac(vol, -0.020089285714285716, K[30]);
    K[31] = Ops::fmac(vol, -0.020089285714285716, K[31]);
    K[32] = Ops::fmac(vol, -0.008035714285714285, K[32]);
    K[33] = Ops::fmac(vol, 0.024107142857142858, K[33]);
    K[34] = Ops::fmac(vol, 0.08035714285714286, K[34]);
    K[35] = Ops::fmac(vol, -0.020089285714285716, K[35]);
    K[36] = Ops::fmac(vol, -0.008035714285714285, K[36]);
    K[37] = Ops::fmac(vol, 0.04017857142857143, K[37]);
    K[38] = Ops::fmac(vol, -0.020089285714285716, K[38]);
    K[39] = Ops::fmac(vol, 0.024107142857142858, K[39]);
    K[40] = Ops::fmac(vol, 0.08035714285714286, K[40]);
    K[41] = Ops::fmac(vol, -0.028125, K[41]);
    K[42] = Ops::fmac(vol, -0.008035714285714285, K[42]);
    K[43] = Ops::fmac(vol, -0.020089285714285716, K[43]);
    K[44] = Ops::fmac(vol, 0.024107142857142858, K[44]);
    K[45] = Ops::fmac(vol, 0.08035714285714286, K[45]);
    K[46] = Ops::fmac(vol, -0.020089285714285716, K[46]);
    K[47] = Ops::fmac(vol, 0.04017857142857143, K[47]);
    K[48] = Ops::fmac(vol, 0.024107142857142858, K[48]);
    K[49] = Ops::fmac(vol, 0.08035714285714286, K[49]);
    K[50] = Ops::fmac(vol, -0.028125, K[50]);
    K[51] = Ops::fmac(vol, 0.024107142857142858, K[51]);
    K[52] = Ops::fmac(vol, 0.08035714285714286, K[52]);
    K[53] = Ops::fmac(vol, 0.024107142857142858, K[53]);
    K[54] = Ops::fmac(vol, 0.2892857142857143, K[54]);
  }
  template <class Ops> __device__ __forceinline__ static void mass_upper(const typename Ops::T& vol, typename Ops::T* K) {
    K[0] = Ops::mulc(vol, 0.01130952380952381);
    K[1] = Ops::mulc(vol, 0.001636904761904762);
    K[2] = Ops::mulc(vol, 0.001636904761904762);
    K[3] = Ops::mulc(vol, 0.0026785714285714286);
    K[4] = Ops::mulc(vol, 0.0);
    K[5] = Ops::mulc(vol, 0.0026785714285714286);
    K[6] = Ops::mulc(vol, 0.0);
    K[7] = Ops::mulc(vol, 0.0040178571428571425);
    K[8] = Ops::mulc(vol, 0.0040178571428571425);
    K[9] = Ops::mulc(vol, 0.005357142857142857);
    K[10] = Ops::mulc(vol, 0.01130952380952381);
    K[11] = Ops::mulc(vol, 0.001636904761904762);
    K[12] = Ops::mulc(vol, 0.0);
    K[13] = Ops::mulc(vol, 0.0026785714285714286);
    K[14] = Ops::mulc(vol, 0.0040178571428571425);
    K[15] = Ops::mulc(vol, 0.0040178571428571425);
    K[16] = Ops::mulc(vol, 0.0026785714285714286);
    K[17] = Ops::mulc(vol, 0.0);
    K[18] = Ops::mulc(vol, 0.005357142857142857);
    K[19] = Ops::mulc(vol, 0.01130952380952381);
    K[20] = Ops::mulc(vol, 0.0040178571428571425);
    K[21] = Ops::mulc(vol, 0.0040178571428571425);
    K[22] = Ops::mulc(vol, 0.0);
    K[23] = Ops::mulc(vol, 0.0026785714285714286);
    K[24] = Ops::mulc(vol, 0.0);
    K[25] = Ops::mulc(vol, 0.0026785714285714286);
    K[26] = Ops::mulc(vol, 0.005357142857142857);
    K[27] = Ops::mulc(vol, 0.08035714285714286);
    K[28] = Ops::mulc(vol, -0.028125);
    K[29] = Ops::mulc(vol, 0.04017857142857143);
    K[30] = Ops::mulc(vol, -0.020089285714285716);
    K[31] = Ops::mulc(vol, -0.020089285714285716);
    K[32] = Ops::mulc(vol, -0.008035714285714285);
    K[33] = Ops::mulc(vol, 0.024107142857142858);
    K[34] = Ops::mulc(vol, 0.08035714285714286);
    K[35] = Ops::mulc(vol, -0.020089285714285716);
    K[36] = Ops::mulc(vol, -0.008035714285714285);
    K[37] = Ops::mulc(vol, 0.04017857142857143);
    K[38] = Ops::mulc(vol, -0.020089285714285716);
    K[39] = Ops::mulc(vol, 0.024107142857142858);
    K[40] = Ops::mulc(vol, 0.08035714285714286);
    K[41] = Ops::mulc(vol, -0.028125);
    K[42] = Ops::mulc(vol, -0.008035714285714285);
    K[43] = Ops::mulc(vol, -0.020089285714285716);
    K[44] = Ops::mulc(vol, 0.024107142857142858);
    K[45] = Ops::mulc(vol, 0.08035714285714286);
    K[46] = Ops::mulc(vol, -0.020089285714285716);
    K[47] = Ops::mulc(vol, 0.04017857142857143);
    K[48] = Ops::mulc(vol, 0.024107142857142858);
    K[49] = Ops::mulc(vol, 0.08035714285714286);
    K[50] = Ops::mulc(vol, -0.028125);
    K[51] = Ops::mulc(vol, 0.024107142857142858);
    K[52] = Ops::mulc(vol, 0.08035714285714286);
    K[53] = Ops::mulc(vol, 0.024107142857142858);
    K[54] = Ops::mulc(vol, 0.2892857142857143);
  }
  template <class Ops, bool STIFF, bool MASS> __device__ __forceinline__ static void action_upper(const typename Ops::T* Lam, const typename Ops::T& vol, const typename Ops::T* x, typename Ops::T* y) {
    typename Ops::T k;
    { if constexpr (STIFF) { k = Ops::mulc(Lam[0], 0.85); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, 0.01130952380952381, k); } y[0] = Ops::fma3(k, x[0], y[0]); }
    { if constexpr (STIFF) { k = Ops::mulc(Lam[1], 0.175); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, 0.001636904761904762, k); } y[0] = Ops::fma3(k, x[1], y[0]); y[1] = Ops::fma3(k, x[0], y[1]); }
    { if constexpr (STIFF) { k = Ops::mulc(Lam[2], 0.175); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, 0.001636904761904762, k); } y[0] = Ops::fma3(k, x[2], y[0]); y[2] = Ops::fma3(k, x[0], y[2]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[1], 1.425, Ops::mulc(Lam[0], 0.075)); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, 0.0026785714285714286, k); } y[0] = Ops::fma3(k, x[3], y[0]); y[3] = Ops::fma3(k, x[0], y[3]); }
    if constexpr (STIFF) { if constexpr (STIFF) { k = Ops::fmac(Lam[1], -0.6, Ops::mulc(Lam[0], 0.075)); } else { k = Ops::zero(); } y[0] = Ops::fma3(k, x[4], y[0]); y[4] = Ops::fma3(k, x[0], y[4]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[2], 1.425, Ops::mulc(Lam[0], 0.075)); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, 0.0026785714285714286, k); } y[0] = Ops::fma3(k, x[5], y[0]); y[5] = Ops::fma3(k, x[0], y[5]); }
    if constexpr (STIFF) { if constexpr (STIFF) { k = Ops::fmac(Lam[2], -0.6, Ops::mulc(Lam[0], 0.075)); } else { k = Ops::zero(); } y[0] = Ops::fma3(k, x[6], y[0]); y[6] = Ops::fma3(k, x[0], y[6]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[2], 0.075, Ops::mulc(Lam[1], 0.075)); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, 0.0040178571428571425, k); } y[0] = Ops::fma3(k, x[7], y[0]); y[7] = Ops::fma3(k, x[0], y[7]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[2], 0.075, Ops::mulc(Lam[1], 0.075)); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, 0.0040178571428571425, k); } y[0] = Ops::fma3(k, x[8], y[0]); y[8] = Ops::fma3(k, x[0], y[8]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[2], 0.225, Ops::fmac(Lam[1], 0.225, Ops::mulc(Lam[0], 0.225))); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, 0.005357142857142857, k); } y[0] = Ops::fma3(k, x[9], y[0]); y[9] = Ops::fma3(k, x[0], y[9]); }
    { if constexpr (STIFF) { k = Ops::mulc(Lam[3], 0.85); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, 0.01130952380952381, k); } y[1] = Ops::fma3(k, x[1], y[1]); }
    { if constexpr (STIFF) { k = Ops::mulc(Lam[4], 0.175); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, 0.001636904761904762, k); } y[1] = Ops::fma3(k, x[2], y[1]); y[2] = Ops::fma3(k, x[1], y[2]); }
    if constexpr (STIFF) { if constexpr (STIFF) { k = Ops::fmac(Lam[3], 0.075, Ops::mulc(Lam[1], -0.6)); } else { k = Ops::zero(); } y[1] = Ops::fma3(k, x[3], y[1]); y[3] = Ops::fma3(k, x[1], y[3]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[3], 0.075, Ops::mulc(Lam[1], 1.425)); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, 0.0026785714285714286, k); } y[1] = Ops::fma3(k, x[4], y[1]); y[4] = Ops::fma3(k, x[1], y[4]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[4], 0.075, Ops::mulc(Lam[1], 0.075)); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, 0.0040178571428571425, k); } y[1] = Ops::fma3(k, x[5], y[1]); y[5] = Ops::fma3(k, x[1], y[5]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[4], 0.075, Ops::mulc(Lam[1], 0.075)); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, 0.0040178571428571425, k); } y[1] = Ops::fma3(k, x[6], y[1]); y[6] = Ops::fma3(k, x[1], y[6]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[4], 1.425, Ops::mulc(Lam[3], 0.075)); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, 0.0026785714285714286, k); } y[1] = Ops::fma3(k, x[7], y[1]); y[7] = Ops::fma3(k, x[1], y[7]); }
    if constexpr (STIFF) { if constexpr (STIFF) { k = Ops::fmac(Lam[4], -0.6, Ops::mulc(Lam[3], 0.075)); } else { k = Ops::zero(); } y[1] = Ops::fma3(k, x[8], y[1]); y[8] = Ops::fma3(k, x[1], y[8]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[4], 0.225, Ops::fmac(Lam[3], 0.225, Ops::mulc(Lam[1], 0.225))); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, 0.005357142857142857, k); } y[1] = Ops::fma3(k, x[9], y[1]); y[9] = Ops::fma3(k, x[1], y[9]); }
    { if constexpr (STIFF) { k = Ops::mulc(Lam[5], 0.85); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, 0.01130952380952381, k); } y[2] = Ops::fma3(k, x[2], y[2]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[4], 0.075, Ops::mulc(Lam[2], 0.075)); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, 0.0040178571428571425, k); } y[2] = Ops::fma3(k, x[3], y[2]); y[3] = Ops::fma3(k, x[2], y[3]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[4], 0.075, Ops::mulc(Lam[2], 0.075)); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, 0.0040178571428571425, k); } y[2] = Ops::fma3(k, x[4], y[2]); y[4] = Ops::fma3(k, x[2], y[4]); }
    if constexpr (STIFF) { if constexpr (STIFF) { k = Ops::fmac(Lam[5], 0.075, Ops::mulc(Lam[2], -0.6)); } else { k = Ops::zero(); } y[2] = Ops::fma3(k, x[5], y[2]); y[5] = Ops::fma3(k, x[2], y[5]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[5], 0.075, Ops::mulc(Lam[2], 1.425)); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, 0.0026785714285714286, k); } y[2] = Ops::fma3(k, x[6], y[2]); y[6] = Ops::fma3(k, x[2], y[6]); }
    if constexpr (STIFF) { if constexpr (STIFF) { k = Ops::fmac(Lam[5], 0.075, Ops::mulc(Lam[4], -0.6)); } else { k = Ops::zero(); } y[2] = Ops::fma3(k, x[7], y[2]); y[7] = Ops::fma3(k, x[2], y[7]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[5], 0.075, Ops::mulc(Lam[4], 1.425)); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, 0.0026785714285714286, k); } y[2] = Ops::fma3(k, x[8], y[2]); y[8] = Ops::fma3(k, x[2], y[8]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[5], 0.225, Ops::fmac(Lam[4], 0.225, Ops::mulc(Lam[2], 0.225))); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, 0.005357142857142857, k); } y[2] = Ops::fma3(k, x[9], y[2]); y[9] = Ops::fma3(k, x[2], y[9]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[3], 3.375, Ops::fmac(Lam[1], 3.375, Ops::mulc(Lam[0], 3.375))); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, 0.08035714285714286, k); } y[3] = Ops::fma3(k, x[3], y[3]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[3], -0.675, Ops::fmac(Lam[1], 1.35, Ops::mulc(Lam[0], -0.675))); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, -0.028125, k); } y[3] = Ops::fma3(k, x[4], y[3]); y[4] = Ops::fma3(k, x[3], y[4]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[4], 3.375, Ops::fmac(Lam[2], 1.6875, Ops::fmac(Lam[1], 1.6875, Ops::mulc(Lam[0], 1.6875)))); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, 0.04017857142857143, k); } y[3] = Ops::fma3(k, x[5], y[3]); y[5] = Ops::fma3(k, x[3], y[5]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[4], -0.675, Ops::fmac(Lam[2], -0.3375, Ops::fmac(Lam[1], -0.3375, Ops::mulc(Lam[0], -0.3375)))); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, -0.020089285714285716, k); } y[3] = Ops::fma3(k, x[6], y[3]); y[6] = Ops::fma3(k, x[3], y[6]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[4], -0.3375, Ops::fmac(Lam[3], -0.3375, Ops::fmac(Lam[2], -0.675, Ops::mulc(Lam[1], -0.3375)))); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, -0.020089285714285716, k); } y[3] = Ops::fma3(k, x[7], y[3]); y[7] = Ops::fma3(k, x[3], y[7]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[4], -0.3375, Ops::fmac(Lam[3], -0.3375, Ops::fmac(Lam[2], -0.675, Ops::mulc(Lam[1], -0.3375)))); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, -0.008035714285714285, k); } y[3] = Ops::fma3(k, x[8], y[3]); y[8] = Ops::fma3(k, x[3], y[8]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[4], 2.025, Ops::fmac(Lam[3], 2.025, Ops::fmac(Lam[2], 4.05, Ops::mulc(Lam[1], 2.025)))); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, 0.024107142857142858, k); } y[3] = Ops::fma3(k, x[9], y[3]); y[9] = Ops::fma3(k, x[3], y[9]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[3], 3.375, Ops::fmac(Lam[1], 3.375, Ops::mulc(Lam[0], 3.375))); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, 0.08035714285714286, k); } y[4] = Ops::fma3(k, x[4], y[4]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[4], -0.675, Ops::fmac(Lam[2], -0.3375, Ops::fmac(Lam[1], -0.3375, Ops::mulc(Lam[0], -0.3375)))); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, -0.020089285714285716, k); } y[4] = Ops::fma3(k, x[5], y[4]); y[5] = Ops::fma3(k, x[4], y[5]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[4], -0.675, Ops::fmac(Lam[2], -0.3375, Ops::fmac(Lam[1], -0.3375, Ops::mulc(Lam[0], -0.3375)))); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, -0.008035714285714285, k); } y[4] = Ops::fma3(k, x[6], y[4]); y[6] = Ops::fma3(k, x[4], y[6]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[4], 1.6875, Ops::fmac(Lam[3], 1.6875, Ops::fmac(Lam[2], 3.375, Ops::mulc(Lam[1], 1.6875)))); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, 0.04017857142857143, k); } y[4] = Ops::fma3(k, x[7], y[4]); y[7] = Ops::fma3(k, x[4], y[7]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[4], -0.3375, Ops::fmac(Lam[3], -0.3375, Ops::fmac(Lam[2], -0.675, Ops::mulc(Lam[1], -0.3375)))); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, -0.020089285714285716, k); } y[4] = Ops::fma3(k, x[8], y[4]); y[8] = Ops::fma3(k, x[4], y[8]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[4], 4.05, Ops::fmac(Lam[2], 2.025, Ops::fmac(Lam[1], 2.025, Ops::mulc(Lam[0], 2.025)))); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, 0.024107142857142858, k); } y[4] = Ops::fma3(k, x[9], y[4]); y[9] = Ops::fma3(k, x[4], y[9]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[5], 3.375, Ops::fmac(Lam[2], 3.375, Ops::mulc(Lam[0], 3.375))); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, 0.08035714285714286, k); } y[5] = Ops::fma3(k, x[5], y[5]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[5], -0.675, Ops::fmac(Lam[2], 1.35, Ops::mulc(Lam[0], -0.675))); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, -0.028125, k); } y[5] = Ops::fma3(k, x[6], y[5]); y[6] = Ops::fma3(k, x[5], y[6]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[5], -0.3375, Ops::fmac(Lam[4], -0.3375, Ops::fmac(Lam[2], -0.3375, Ops::mulc(Lam[1], -0.675)))); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, -0.008035714285714285, k); } y[5] = Ops::fma3(k, x[7], y[5]); y[7] = Ops::fma3(k, x[5], y[7]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[5], -0.3375, Ops::fmac(Lam[4], -0.3375, Ops::fmac(Lam[2], -0.3375, Ops::mulc(Lam[1], -0.675)))); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, -0.020089285714285716, k); } y[5] = Ops::fma3(k, x[8], y[5]); y[8] = Ops::fma3(k, x[5], y[8]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[5], 2.025, Ops::fmac(Lam[4], 2.025, Ops::fmac(Lam[2], 2.025, Ops::mulc(Lam[1], 4.05)))); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, 0.024107142857142858, k); } y[5] = Ops::fma3(k, x[9], y[5]); y[9] = Ops::fma3(k, x[5], y[9]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[5], 3.375, Ops::fmac(Lam[2], 3.375, Ops::mulc(Lam[0], 3.375))); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, 0.08035714285714286, k); } y[6] = Ops::fma3(k, x[6], y[6]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[5], -0.3375, Ops::fmac(Lam[4], -0.3375, Ops::fmac(Lam[2], -0.3375, Ops::mulc(Lam[1], -0.675)))); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, -0.020089285714285716, k); } y[6] = Ops::fma3(k, x[7], y[6]); y[7] = Ops::fma3(k, x[6], y[7]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[5], 1.6875, Ops::fmac(Lam[4], 1.6875, Ops::fmac(Lam[2], 1.6875, Ops::mulc(Lam[1], 3.375)))); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, 0.04017857142857143, k); } y[6] = Ops::fma3(k, x[8], y[6]); y[8] = Ops::fma3(k, x[6], y[8]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[4], 4.05, Ops::fmac(Lam[2], 2.025, Ops::fmac(Lam[1], 2.025, Ops::mulc(Lam[0], 2.025)))); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, 0.024107142857142858, k); } y[6] = Ops::fma3(k, x[9], y[6]); y[9] = Ops::fma3(k, x[6], y[9]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[5], 3.375, Ops::fmac(Lam[4], 3.375, Ops::mulc(Lam[3], 3.375))); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, 0.08035714285714286, k); } y[7] = Ops::fma3(k, x[7], y[7]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[5], -0.675, Ops::fmac(Lam[4], 1.35, Ops::mulc(Lam[3], -0.675))); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, -0.028125, k); } y[7] = Ops::fma3(k, x[8], y[7]); y[8] = Ops::fma3(k, x[7], y[8]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[5], 2.025, Ops::fmac(Lam[4], 2.025, Ops::fmac(Lam[2], 2.025, Ops::mulc(Lam[1], 4.05)))); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, 0.024107142857142858, k); } y[7] = Ops::fma3(k, x[9], y[7]); y[9] = Ops::fma3(k, x[7], y[9]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[5], 3.375, Ops::fmac(Lam[4], 3.375, Ops::mulc(Lam[3], 3.375))); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, 0.08035714285714286, k); } y[8] = Ops::fma3(k, x[8], y[8]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[4], 2.025, Ops::fmac(Lam[3], 2.025, Ops::fmac(Lam[2], 4.05, Ops::mulc(Lam[1], 2.025)))); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, 0.024107142857142858, k); } y[8] = Ops::fma3(k, x[9], y[8]); y[9] = Ops::fma3(k, x[8], y[9]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[5], 8.1, Ops::fmac(Lam[4], 8.1, Ops::fmac(Lam[3], 8.1, Ops::fmac(Lam[2], 8.1, Ops::fmac(Lam[1], 8.1, Ops::mulc(Lam[0], 8.1)))))); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, 0.2892857142857143, k); } y[9] = Ops::fma3(k, x[9], y[9]); }
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
  template <class Ops> __device__ __forceinline__ static void stiffness_upper(const typename Ops::T* Lam, typename Ops::T* K) {
    K[0] = Ops::mulc(Lam[0], 0.746031746031746);
    K[1] = Ops::mulc(Lam[1], -0.11322751322751323);
    K[2] = Ops::mulc(Lam[2], -0.11322751322751323);
    K[3] = Ops::fmac(Lam[1], 1.5576719576719578, Ops::mulc(Lam[0], 0.25396825396825395));
    K[4] = Ops::fmac(Lam[1], -0.8507936507936508, Ops::mulc(Lam[0], 0.08465608465608465));
    K[5] = Ops::fmac(Lam[1], 0.40634920634920635, Ops::mulc(Lam[0], -0.08465608465608465));
    K[6] = Ops::fmac(Lam[2], 1.5576719576719578, Ops::mulc(Lam[0], 0.25396825396825395));
    K[7] = Ops::fmac(Lam[2], -0.8507936507936508, Ops::mulc(Lam[0], 0.08465608465608465));
    K[8] = Ops::fmac(Lam[2], 0.40634920634920635, Ops::mulc(Lam[0], -0.08465608465608465));
    K[9] = Ops::fmac(Lam[2], -0.08465608465608465, Ops::mulc(Lam[1], -0.08465608465608465));
    K[10] = Ops::fmac(Lam[2], -0.08465608465608465, Ops::mulc(Lam[1], -0.08465608465608465));
    K[11] = Ops::fmac(Lam[2], -0.08465608465608465, Ops::mulc(Lam[1], -0.08465608465608465));
    K[12] = Ops::fmac(Lam[2], 0.6349206349206349, Ops::fmac(Lam[1], 0.6349206349206349, Ops::mulc(Lam[0], 0.4656084656084656)));
    K[13] = Ops::fmac(Lam[2], -0.042328042328042326, Ops::fmac(Lam[1], -0.042328042328042326, Ops::mulc(Lam[0], -0.21164021164021163)));
    K[14] = Ops::fmac(Lam[2], -0.042328042328042326, Ops::fmac(Lam[1], -0.042328042328042326, Ops::mulc(Lam[0], -0.21164021164021163)));
    K[15] = Ops::mulc(Lam[3], 0.746031746031746);
    K[16] = Ops::mulc(Lam[4], -0.11322751322751323);
    K[17] = Ops::fmac(Lam[3], -0.08465608465608465, Ops::mulc(Lam[1], 0.40634920634920635));
    K[18] = Ops::fmac(Lam[3], 0.08465608465608465, Ops::mulc(Lam[1], -0.8507936507936508));
    K[19] = Ops::fmac(Lam[3], 0.25396825396825395, Ops::mulc(Lam[1], 1.5576719576719578));
    K[20] = Ops::fmac(Lam[4], -0.08465608465608465, Ops::mulc(Lam[1], -0.08465608465608465));
    K[21] = Ops::fmac(Lam[4], -0.08465608465608465, Ops::mulc(Lam[1], -0.08465608465608465));
    K[22] = Ops::fmac(Lam[4], -0.08465608465608465, Ops::mulc(Lam[1], -0.08465608465608465));
    K[23] = Ops::fmac(Lam[4], 1.5576719576719578, Ops::mulc(Lam[3], 0.25396825396825395));
    K[24] = Ops::fmac(Lam[4], -0.8507936507936508, Ops::mulc(Lam[3], 0.08465608465608465));
    K[25] = Ops::fmac(Lam[4], 0.40634920634920635, Ops::mulc(Lam[3], -0.08465608465608465));
    K[26] = Ops::fmac(Lam[4], -0.042328042328042326, Ops::fmac(Lam[3], -0.21164021164021163, Ops::mulc(Lam[1], -0.042328042328042326)));
    K[27] = Ops::fmac(Lam[4], 0.6349206349206349, Ops::fmac(Lam[3], 0.4656084656084656, Ops::mulc(Lam[1], 0.6349206349206349)));
    K[28] = Ops::fmac(Lam[4], -0.042328042328042326, Ops::fmac(Lam[3], -0.21164021164021163, Ops::mulc(Lam[1], -0.042328042328042326)));
    K[29] = Ops::mulc(Lam[5], 0.746031746031746);
    K[30] = Ops::fmac(Lam[4], -0.08465608465608465, Ops::mulc(Lam[2], -0.08465608465608465));
    K[31] = Ops::fmac(Lam[4], -0.08465608465608465, Ops::mulc(Lam[2], -0.08465608465608465));
    K[32] = Ops::fmac(Lam[4], -0.08465608465608465, Ops::mulc(Lam[2], -0.08465608465608465));
    K[33] = Ops::fmac(Lam[5], -0.08465608465608465, Ops::mulc(Lam[2], 0.40634920634920635));
    K[34] = Ops::fmac(Lam[5], 0.08465608465608465, Ops::mulc(Lam[2], -0.8507936507936508));
    K[35] = Ops::fmac(Lam[5], 0.25396825396825395, Ops::mulc(Lam[2], 1.5576719576719578));
    K[36] = Ops::fmac(Lam[5], -0.08465608465608465, Ops::mulc(Lam[4], 0.40634920634920635));
    K[37] = Ops::fmac(Lam[5], 0.08465608465608465, Ops::mulc(Lam[4], -0.8507936507936508));
    K[38] = Ops::fmac(Lam[5], 0.25396825396825395, Ops::mulc(Lam[4], 1.5576719576719578));
    K[39] = Ops::fmac(Lam[5], -0.21164021164021163, Ops::fmac(Lam[4], -0.042328042328042326, Ops::mulc(Lam[2], -0.042328042328042326)));
    K[40] = Ops::fmac(Lam[5], -0.21164021164021163, Ops::fmac(Lam[4], -0.042328042328042326, Ops::mulc(Lam[2], -0.042328042328042326)));
    K[41] = Ops::fmac(Lam[5], 0.4656084656084656, Ops::fmac(Lam[4], 0.6349206349206349, Ops::mulc(Lam[2], 0.6349206349206349)));
    K[42] = Ops::fmac(Lam[3], 4.1989417989417985, Ops::fmac(Lam[1], 4.1989417989417985, Ops::mulc(Lam[0], 3.657142857142857)));
    K[43] = Ops::fmac(Lam[3], -1.5238095238095237, Ops::fmac(Lam[1], 1.0497354497354496, Ops::mulc(Lam[0], -1.3206349206349206)));
    K[44] = Ops::fmac(Lam[3], 0.6772486772486772, Ops::fmac(Lam[1], -0.6772486772486772, Ops::mulc(Lam[0], 0.6772486772486772)));
    K[45] = Ops::fmac(Lam[4], 4.1989417989417985, Ops::fmac(Lam[2], 2.0994708994708993, Ops::fmac(Lam[1], 2.0994708994708993, Ops::mulc(Lam[0], 1.8285714285714285))));
    K[46] = Ops::fmac(Lam[4], -1.5238095238095237, Ops::fmac(Lam[2], -0.9312169312169312, Ops::fmac(Lam[1], -0.5925925925925926, Ops::mulc(Lam[0], -0.728042328042328))));
    K[47] = Ops::fmac(Lam[4], 0.6772486772486772, Ops::fmac(Lam[2], 0.4740740740740741, Ops::fmac(Lam[1], 0.20317460317460317, Ops::mulc(Lam[0], 0.20317460317460317))));
    K[48] = Ops::fmac(Lam[4], 0.20317460317460317, Ops::fmac(Lam[3], 0.20317460317460317, Ops::fmac(Lam[2], 0.6772486772486772, Ops::mulc(Lam[1], 0.4740740740740741))));
    K[49] = Ops::fmac(Lam[4], 0.08465608465608465, Ops::fmac(Lam[3], 0.08465608465608465, Ops::fmac(Lam[2], 0.3047619047619048, Ops::mulc(Lam[1], 0.2201058201058201))));
    K[50] = Ops::fmac(Lam[4], 0.20317460317460317, Ops::fmac(Lam[3], 0.20317460317460317, Ops::fmac(Lam[2], 0.40634920634920635, Ops::mulc(Lam[1], 0.20317460317460317))));
    K[51] = Ops::fmac(Lam[4], 3.250793650793651, Ops::fmac(Lam[3], 3.250793650793651, Ops::fmac(Lam[2], 5.147089947089947, Ops::fmac(Lam[1], 3.250793650793651, Ops::mulc(Lam[0], 0.2708994708994709)))));
    K[52] = Ops::fmac(Lam[4], -0.5417989417989418, Ops::fmac(Lam[3], -0.5417989417989418, Ops::fmac(Lam[2], -0.8126984126984127, Ops::mulc(Lam[0], 0.8126984126984127))));
    K[53] = Ops::fmac(Lam[4], -0.5417989417989418, Ops::fmac(Lam[3], -0.5417989417989418, Ops::fmac(Lam[2], -1.3544973544973544, Ops::fmac(Lam[1], -0.5417989417989418, Ops::mulc(Lam[0], 0.2708994708994709)))));
    K[54] = Ops::fmac(Lam[3], 4.901587301587302, Ops::fmac(Lam[1], 3.8857142857142857, Ops::mulc(Lam[0], 4.901587301587302)));
    K[55] = Ops::fmac(Lam[3], -1.3206349206349206, Ops::fmac(Lam[1], 1.0497354497354496, Ops::mulc(Lam[0], -1.5238095238095237)));
    K[56] = Ops::fmac(Lam[4], -1.5238095238095237, Ops::fmac(Lam[2], -0.5925925925925926, Ops::fmac(Lam[1], -0.9312169312169312, Ops::mulc(Lam[0], -0.728042328042328))));
    K[57] = Ops::fmac(Lam[4], -0.7873015873015873, Ops::fmac(Lam[2], -0.39365079365079364, Ops::fmac(Lam[1], -0.39365079365079364, Ops::mulc(Lam[0], -0.2920634920634921))));
    K[58] = Ops::fmac(Lam[4], 0.3047619047619048, Ops::fmac(Lam[2], 0.2201058201058201, Ops::fmac(Lam[1], 0.08465608465608465, Ops::mulc(Lam[0], 0.08465608465608465))));
    K[59] = Ops::fmac(Lam[4], -0.5925925925925926, Ops::fmac(Lam[3], -0.728042328042328, Ops::fmac(Lam[2], -1.5238095238095237, Ops::mulc(Lam[1], -0.9312169312169312))));
    K[60] = Ops::fmac(Lam[4], -0.39365079365079364, Ops::fmac(Lam[3], -0.2920634920634921, Ops::fmac(Lam[2], -0.7873015873015873, Ops::mulc(Lam[1], -0.39365079365079364))));
    K[61] = Ops::fmac(Lam[4], 0.2201058201058201, Ops::fmac(Lam[3], 0.08465608465608465, Ops::fmac(Lam[2], 0.3047619047619048, Ops::mulc(Lam[1], 0.08465608465608465))));
    K[62] = Ops::fmac(Lam[4], 4.673015873015873, Ops::fmac(Lam[3], -1.0158730158730158, Ops::fmac(Lam[2], 1.8285714285714285, Ops::fmac(Lam[1], 1.8285714285714285, Ops::mulc(Lam[0], 2.641269841269841)))));
    K[63] = Ops::fmac(Lam[4], 1.8285714285714285, Ops::fmac(Lam[3], 2.641269841269841, Ops::fmac(Lam[2], 4.673015873015873, Ops::fmac(Lam[1], 1.8285714285714285, Ops::mulc(Lam[0], -1.0158730158730158)))));
    K[64] = Ops::fmac(Lam[4], -1.4222222222222223, Ops::fmac(Lam[3], -0.6095238095238096, Ops::fmac(Lam[2], -1.4222222222222223, Ops::fmac(Lam[1], -1.0158730158730158, Ops::mulc(Lam[0], -0.6095238095238096)))));
    K[65] = Ops::fmac(Lam[3], 3.657142857142857, Ops::fmac(Lam[1], 4.1989417989417985, Ops::mulc(Lam[0], 4.1989417989417985)));
    K[66] = Ops::fmac(Lam[4], 0.6772486772486772, Ops::fmac(Lam[2], 0.20317460317460317, Ops::fmac(Lam[1], 0.4740740740740741, Ops::mulc(Lam[0], 0.20317460317460317))));
    K[67] = Ops::fmac(Lam[4], 0.3047619047619048, Ops::fmac(Lam[2], 0.08465608465608465, Ops::fmac(Lam[1], 0.2201058201058201, Ops::mulc(Lam[0], 0.08465608465608465))));
    K[68] = Ops::fmac(Lam[4], 0.40634920634920635, Ops::fmac(Lam[2], 0.20317460317460317, Ops::fmac(Lam[1], 0.20317460317460317, Ops::mulc(Lam[0], 0.20317460317460317))));
    K[69] = Ops::fmac(Lam[4], 2.0994708994708993, Ops::fmac(Lam[3], 1.8285714285714285, Ops::fmac(Lam[2], 4.1989417989417985, Ops::mulc(Lam[1], 2.0994708994708993))));
    K[70] = Ops::fmac(Lam[4], -0.9312169312169312, Ops::fmac(Lam[3], -0.728042328042328, Ops::fmac(Lam[2], -1.5238095238095237, Ops::mulc(Lam[1], -0.5925925925925926))));
    K[71] = Ops::fmac(Lam[4], 0.4740740740740741, Ops::fmac(Lam[3], 0.20317460317460317, Ops::fmac(Lam[2], 0.6772486772486772, Ops::mulc(Lam[1], 0.20317460317460317))));
    K[72] = Ops::fmac(Lam[4], -0.8126984126984127, Ops::fmac(Lam[3], 0.8126984126984127, Ops::fmac(Lam[2], -0.5417989417989418, Ops::mulc(Lam[0], -0.5417989417989418))));
    K[73] = Ops::fmac(Lam[4], 5.147089947089947, Ops::fmac(Lam[3], 0.2708994708994709, Ops::fmac(Lam[2], 3.250793650793651, Ops::fmac(Lam[1], 3.250793650793651, Ops::mulc(Lam[0], 3.250793650793651)))));
    K[74] = Ops::fmac(Lam[4], -1.3544973544973544, Ops::fmac(Lam[3], 0.2708994708994709, Ops::fmac(Lam[2], -0.5417989417989418, Ops::fmac(Lam[1], -0.5417989417989418, Ops::mulc(Lam[0], -0.5417989417989418)))));
    K[75] = Ops::fmac(Lam[5], 4.1989417989417985, Ops::fmac(Lam[2], 4.1989417989417985, Ops::mulc(Lam[0], 3.657142857142857)));
    K[76] = Ops::fmac(Lam[5], -1.5238095238095237, Ops::fmac(Lam[2], 1.0497354497354496, Ops::mulc(Lam[0], -1.3206349206349206)));
    K[77] = Ops::fmac(Lam[5], 0.6772486772486772, Ops::fmac(Lam[2], -0.6772486772486772, Ops::mulc(Lam[0], 0.6772486772486772)));
    K[78] = Ops::fmac(Lam[5], 0.20317460317460317, Ops::fmac(Lam[4], 0.20317460317460317, Ops::fmac(Lam[2], 0.20317460317460317, Ops::mulc(Lam[1], 0.40634920634920635))));
    K[79] = Ops::fmac(Lam[5], 0.08465608465608465, Ops::fmac(Lam[4], 0.08465608465608465, Ops::fmac(Lam[2], 0.2201058201058201, Ops::mulc(Lam[1], 0.3047619047619048))));
    K[80] = Ops::fmac(Lam[5], 0.20317460317460317, Ops::fmac(Lam[4], 0.20317460317460317, Ops::fmac(Lam[2], 0.4740740740740741, Ops::mulc(Lam[1], 0.6772486772486772))));
    K[81] = Ops::fmac(Lam[5], 3.250793650793651, Ops::fmac(Lam[4], 3.250793650793651, Ops::fmac(Lam[2], 3.250793650793651, Ops::fmac(Lam[1], 5.147089947089947, Ops::mulc(Lam[0], 0.2708994708994709)))));
    K[82] = Ops::fmac(Lam[5], -0.5417989417989418, Ops::fmac(Lam[4], -0.5417989417989418, Ops::fmac(Lam[2], -0.5417989417989418, Ops::fmac(Lam[1], -1.3544973544973544, Ops::mulc(Lam[0], 0.2708994708994709)))));
    K[83] = Ops::fmac(Lam[5], -0.5417989417989418, Ops::fmac(Lam[4], -0.5417989417989418, Ops::fmac(Lam[1], -0.8126984126984127, Ops::mulc(Lam[0], 0.8126984126984127))));
    K[84] = Ops::fmac(Lam[5], 4.901587301587302, Ops::fmac(Lam[2], 3.8857142857142857, Ops::mulc(Lam[0], 4.901587301587302)));
    K[85] = Ops::fmac(Lam[5], -1.3206349206349206, Ops::fmac(Lam[2], 1.0497354497354496, Ops::mulc(Lam[0], -1.5238095238095237)));
    K[86] = Ops::fmac(Lam[5], 0.08465608465608465, Ops::fmac(Lam[4], 0.2201058201058201, Ops::fmac(Lam[2], 0.08465608465608465, Ops::mulc(Lam[1], 0.3047619047619048))));
    K[87] = Ops::fmac(Lam[5], -0.2920634920634921, Ops::fmac(Lam[4], -0.39365079365079364, Ops::fmac(Lam[2], -0.39365079365079364, Ops::mulc(Lam[1], -0.7873015873015873))));
    K[88] = Ops::fmac(Lam[5], -0.728042328042328, Ops::fmac(Lam[4], -0.5925925925925926, Ops::fmac(Lam[2], -0.9312169312169312, Ops::mulc(Lam[1], -1.5238095238095237))));
    K[89] = Ops::fmac(Lam[5], -1.0158730158730158, Ops::fmac(Lam[4], 4.673015873015873, Ops::fmac(Lam[2], 1.8285714285714285, Ops::fmac(Lam[1], 1.8285714285714285, Ops::mulc(Lam[0], 2.641269841269841)))));
    K[90] = Ops::fmac(Lam[5], -0.6095238095238096, Ops::fmac(Lam[4], -1.4222222222222223, Ops::fmac(Lam[2], -1.0158730158730158, Ops::fmac(Lam[1], -1.4222222222222223, Ops::mulc(Lam[0], -0.6095238095238096)))));
    K[91] = Ops::fmac(Lam[5], 2.641269841269841, Ops::fmac(Lam[4], 1.8285714285714285, Ops::fmac(Lam[2], 1.8285714285714285, Ops::fmac(Lam[1], 4.673015873015873, Ops::mulc(Lam[0], -1.0158730158730158)))));
    K[92] = Ops::fmac(Lam[5], 3.657142857142857, Ops::fmac(Lam[2], 4.1989417989417985, Ops::mulc(Lam[0], 4.1989417989417985)));
    K[93] = Ops::fmac(Lam[5], 0.20317460317460317, Ops::fmac(Lam[4], 0.4740740740740741, Ops::fmac(Lam[2], 0.20317460317460317, Ops::mulc(Lam[1], 0.6772486772486772))));
    K[94] = Ops::fmac(Lam[5], -0.728042328042328, Ops::fmac(Lam[4], -0.9312169312169312, Ops::fmac(Lam[2], -0.5925925925925926, Ops::mulc(Lam[1], -1.5238095238095237))));
    K[95] = Ops::fmac(Lam[5], 1.8285714285714285, Ops::fmac(Lam[4], 2.0994708994708993, Ops::fmac(Lam[2], 2.0994708994708993, Ops::mulc(Lam[1], 4.1989417989417985))));
    K[96] = Ops::fmac(Lam[5], 0.8126984126984127, Ops::fmac(Lam[4], -0.8126984126984127, Ops::fmac(Lam[1], -0.5417989417989418, Ops::mulc(Lam[0], -0.5417989417989418))));
    K[97] = Ops::fmac(Lam[5], 0.2708994708994709, Ops::fmac(Lam[4], -1.3544973544973544, Ops::fmac(Lam[2], -0.5417989417989418, Ops::fmac(Lam[1], -0.5417989417989418, Ops::mulc(Lam[0], -0.5417989417989418)))));
    K[98] = Ops::fmac(Lam[5], 0.2708994708994709, Ops::fmac(Lam[4], 5.147089947089947, Ops::fmac(Lam[2], 3.250793650793651, Ops::fmac(Lam[1], 3.250793650793651, Ops::mulc(Lam[0], 3.250793650793651)))));
    K[99] = Ops::fmac(Lam[5], 4.1989417989417985, Ops::fmac(Lam[4], 4.1989417989417985, Ops::mulc(Lam[3], 3.657142857142857)));
    K[100] = Ops::fmac(Lam[5], -1.5238095238095237, Ops::fmac(Lam[4], 1.0497354497354496, Ops::mulc(Lam[3], -1.3206349206349206)));
    K[101] = Ops::fmac(Lam[5], 0.6772486772486772, Ops::fmac(Lam[4], -0.6772486772486772, Ops::mulc(Lam[3], 0.6772486772486772)));
    K[102] = Ops::fmac(Lam[5], -0.5417989417989418, Ops::fmac(Lam[4], -0.5417989417989418, Ops::fmac(Lam[3], 0.2708994708994709, Ops::fmac(Lam[2], -0.5417989417989418, Ops::mulc(Lam[1], -1.3544973544973544)))));
    K[103] = Ops::fmac(Lam[5], 3.250793650793651, Ops::fmac(Lam[4], 3.250793650793651, Ops::fmac(Lam[3], 0.2708994708994709, Ops::fmac(Lam[2], 3.250793650793651, Ops::mulc(Lam[1], 5.147089947089947)))));
    K[104] = Ops::fmac(Lam[5], -0.5417989417989418, Ops::fmac(Lam[3], 0.8126984126984127, Ops::fmac(Lam[2], -0.5417989417989418, Ops::mulc(Lam[1], -0.8126984126984127))));
    K[105] = Ops::fmac(Lam[5], 4.901587301587302, Ops::fmac(Lam[4], 3.8857142857142857, Ops::mulc(Lam[3], 4.901587301587302)));
    K[106] = Ops::fmac(Lam[5], -1.3206349206349206, Ops::fmac(Lam[4], 1.0497354497354496, Ops::mulc(Lam[3], -1.5238095238095237)));
    K[107] = Ops::fmac(Lam[5], -0.6095238095238096, Ops::fmac(Lam[4], -1.0158730158730158, Ops::fmac(Lam[3], -0.6095238095238096, Ops::fmac(Lam[2], -1.4222222222222223, Ops::mulc(Lam[1], -1.4222222222222223)))));
    K[108] = Ops::fmac(Lam[5], -1.0158730158730158, Ops::fmac(Lam[4], 1.8285714285714285, Ops::fmac(Lam[3], 2.641269841269841, Ops::fmac(Lam[2], 4.673015873015873, Ops::mulc(Lam[1], 1.8285714285714285)))));
    K[109] = Ops::fmac(Lam[5], 2.641269841269841, Ops::fmac(Lam[4], 1.8285714285714285, Ops::fmac(Lam[3], -1.0158730158730158, Ops::fmac(Lam[2], 1.8285714285714285, Ops::mulc(Lam[1], 4.673015873015873)))));
    K[110] = Ops::fmac(Lam[5], 3.657142857142857, Ops::fmac(Lam[4], 4.1989417989417985, Ops::mulc(Lam[3], 4.1989417989417985)));
    K[111] = Ops::fmac(Lam[5], 0.2708994708994709, Ops::fmac(Lam[4], -0.5417989417989418, Ops::fmac(Lam[3], -0.5417989417989418, Ops::fmac(Lam[2], -1.3544973544973544, Ops::mulc(Lam[1], -0.5417989417989418)))));
    K[112] = Ops::fmac(Lam[5], 0.8126984126984127, Ops::fmac(Lam[3], -0.5417989417989418, Ops::fmac(Lam[2], -0.8126984126984127, Ops::mulc(Lam[1], -0.5417989417989418))));
    K[113] = Ops::fmac(Lam[5], 0.2708994708994709, Ops::fmac(Lam[4], 3.250793650793651, Ops::fmac(Lam[3], 3.250793650793651, Ops::fmac(Lam[2], 5.147089947089947, Ops::mulc(Lam[1], 3.250793650793651)))));
    K[114] = Ops::fmac(Lam[5], 11.377777777777778, Ops::fmac(Lam[4], 11.377777777777778, Ops::fmac(Lam[3], 11.377777777777778, Ops::fmac(Lam[2], 11.377777777777778, Ops::fmac(Lam[1], 11.377777777777778, Ops::mulc(Lam[0], 11.377777777777778))))));
    K[115] = Ops::fmac(Lam[5], 1.6253968253968254, Ops::fmac(Lam[4], 1.6253968253968254, Ops::fmac(Lam[3], -1.6253968253968254, Ops::fmac(Lam[2], 1.6253968253968254, Ops::fmac(Lam[1], 4.876190476190477, Ops::mulc(Lam[0], -1.6253968253968254))))));
    K[116] = Ops::fmac(Lam[5], -1.6253968253968254, Ops::fmac(Lam[4], 1.6253968253968254, Ops::fmac(Lam[3], 1.6253968253968254, Ops::fmac(Lam[2], 4.876190476190477, Ops::fmac(Lam[1], 1.6253968253968254, Ops::mulc(Lam[0], -1.6253968253968254))))));
    K[117] = Ops::fmac(Lam[5], 11.377777777777778, Ops::fmac(Lam[4], 11.377777777777778, Ops::fmac(Lam[3], 11.377777777777778, Ops::fmac(Lam[2], 11.377777777777778, Ops::fmac(Lam[1], 11.377777777777778, Ops::mulc(Lam[0], 11.377777777777778))))));
    K[118] = Ops::fmac(Lam[5], -1.6253968253968254, Ops::fmac(Lam[4], 4.876190476190477, Ops::fmac(Lam[3], -1.6253968253968254, Ops::fmac(Lam[2], 1.6253968253968254, Ops::fmac(Lam[1], 1.6253968253968254, Ops::mulc(Lam[0], 1.6253968253968254))))));
    K[119] = Ops::fmac(Lam[5], 11.377777777777778, Ops::fmac(Lam[4], 11.377777777777778, Ops::fmac(Lam[3], 11.377777777777778, Ops::fmac(Lam[2], 11.377777777777778, Ops::fmac(Lam[1], 11.377777777777778, Ops::mulc(Lam[0], 11.377777777777778))))));
  }
  template <class Ops> __device__ __forceinline__ static void mass_upper_add(const typename Ops::T& vol, typename Ops::T* K) {
    K[0] = Ops::fmac(vol, 0.0051146384479717815, K[0]);
    K[1] = Ops::fmac(vol, -0.0004761904761904762, K[1]);
    K[2] = Ops::fmac(vol, -0.0004761904761904762, K[2]);
    K[3] = Ops::fmac(vol, 0.0028218694885361554, K[3]);
    K[4] = Ops::fmac(vol, -0.0014109347442680777, K[4]);
    K[6] = Ops::fmac(vol, 0.0028218694885361554, K[6]);
    K[7] = Ops::fmac(vol, -0.0014109347442680777, K[7]);
    K[9] = Ops::fmac(vol, -0.0019753086419753087, K[9]);
    K[10] = Ops::fmac(vol, -0.00021164021164021165, K[10]);
    K[11] = Ops::fmac(vol, -0.0019753086419753087, K[11]);
    K[12] = Ops::fmac(vol, 0.0028218694885361554, K[12]);
    K[13] = Ops::fmac(vol, -0.0028218694885361554, K[13]);
    K[14] = Ops::fmac(vol, -0.0028218694885361554, K[14]);
    K[15] = Ops::fmac(vol, 0.0051146384479717815, K[15]);
    K[16] = Ops::fmac(vol, -0.0004761904761904762, K[16]);
    K[18] = Ops::fmac(vol, -0.0014109347442680777, K[18]);
    K[19] = Ops::fmac(vol, 0.0028218694885361554, K[19]);
    K[20] = Ops::fmac(vol, -0.0019753086419753087, K[20]);
    K[21] = Ops::fmac(vol, -0.00021164021164021165, K[21]);
    K[22] = Ops::fmac(vol, -0.0019753086419753087, K[22]);
    K[23] = Ops::fmac(vol, 0.0028218694885361554, K[23]);
    K[24] = Ops::fmac(vol, -0.0014109347442680777, K[24]);
    K[26] = Ops::fmac(vol, -0.0028218694885361554, K[26]);
    K[27] = Ops::fmac(vol, 0.0028218694885361554, K[27]);
    K[28] = Ops::fmac(vol, -0.0028218694885361554, K[28]);
    K[29] = Ops::fmac(vol, 0.0051146384479717815, K[29]);
    K[30] = Ops::fmac(vol, -0.0019753086419753087, K[30]);
    K[31] = Ops::fmac(vol, -0.00021164021164021165, K[31]);
    K[32] = Ops::fmac(vol, -0.0019753086419753087, K[32]);
    K[34] = Ops::fmac(vol, -0.0014109347442680777, K[34]);
    K[35] = Ops::fmac(vol, 0.0028218694885361554, K[35]);
    K[37] = Ops::fmac(vol, -0.0014109347442680777, K[37]);
    K[38] = Ops::fmac(vol, 0.0028218694885361554, K[38]);
    K[39] = Ops::fmac(vol, -0.0028218694885361554, K[39]);
    K[40] = Ops::fmac(vol, -0.0028218694885361554, K[40]);
    K[41] = Ops::fmac(vol, 0.0028218694885361554, K[41]);
    K[42] = Ops::fmac(vol, 0.045149911816578486, K[42]);
    K[43] = Ops::fmac(vol, -0.022574955908289243, K[43]);
    K[44] = Ops::fmac(vol, 0.013544973544973546, K[44]);
    K[45] = Ops::fmac(vol, 0.022574955908289243, K[45]);
    K[46] = Ops::fmac(vol, -0.016931216931216932, K[46]);
    K[47] = Ops::fmac(vol, 0.009029982363315696, K[47]);
    K[48] = Ops::fmac(vol, 0.009029982363315696, K[48]);
    K[49] = Ops::fmac(vol, 0.001128747795414462, K[49]);
    K[50] = Ops::fmac(vol, 0.004514991181657848, K[50]);
    K[51] = Ops::fmac(vol, 0.022574955908289243, K[51]);
    K[52] = Ops::fmac(vol, 0.004514991181657848, K[52]);
    K[53] = Ops::fmac(vol, -0.004514991181657848, K[53]);
    K[54] = Ops::fmac(vol, 0.05587301587301587, K[54]);
    K[55] = Ops::fmac(vol, -0.022574955908289243, K[55]);
    K[56] = Ops::fmac(vol, -0.016931216931216932, K[56]);
    K[57] = Ops::fmac(vol, 0.0008465608465608466, K[57]);
    K[58] = Ops::fmac(vol, 0.001128747795414462, K[58]);
    K[59] = Ops::fmac(vol, -0.016931216931216932, K[59]);
    K[60] = Ops::fmac(vol, 0.0008465608465608466, K[60]);
    K[61] = Ops::fmac(vol, 0.001128747795414462, K[61]);
    K[62] = Ops::fmac(vol, 0.006772486772486773, K[62]);
    K[63] = Ops::fmac(vol, 0.006772486772486773, K[63]);
    K[64] = Ops::fmac(vol, -0.013544973544973546, K[64]);
    K[65] = Ops::fmac(vol, 0.045149911816578486, K[65]);
    K[66] = Ops::fmac(vol, 0.009029982363315696, K[66]);
    K[67] = Ops::fmac(vol, 0.001128747795414462, K[67]);
    K[68] = Ops::fmac(vol, 0.004514991181657848, K[68]);
    K[69] = Ops::fmac(vol, 0.022574955908289243, K[69]);
    K[70] = Ops::fmac(vol, -0.016931216931216932, K[70]);
    K[71] = Ops::fmac(vol, 0.009029982363315696, K[71]);
    K[72] = Ops::fmac(vol, 0.004514991181657848, K[72]);
    K[73] = Ops::fmac(vol, 0.022574955908289243, K[73]);
    K[74] = Ops::fmac(vol, -0.004514991181657848, K[74]);
    K[75] = Ops::fmac(vol, 0.045149911816578486, K[75]);
    K[76] = Ops::fmac(vol, -0.022574955908289243, K[76]);
    K[77] = Ops::fmac(vol, 0.013544973544973546, K[77]);
    K[78] = Ops::fmac(vol, 0.004514991181657848, K[78]);
    K[79] = Ops::fmac(vol, 0.001128747795414462, K[79]);
    K[80] = Ops::fmac(vol, 0.009029982363315696, K[80]);
    K[81] = Ops::fmac(vol, 0.022574955908289243, K[81]);
    K[82] = Ops::fmac(vol, -0.004514991181657848, K[82]);
    K[83] = Ops::fmac(vol, 0.004514991181657848, K[83]);
    K[84] = Ops::fmac(vol, 0.05587301587301587, K[84]);
    K[85] = Ops::fmac(vol, -0.022574955908289243, K[85]);
    K[86] = Ops::fmac(vol, 0.001128747795414462, K[86]);
    K[87] = Ops::fmac(vol, 0.0008465608465608466, K[87]);
    K[88] = Ops::fmac(vol, -0.016931216931216932, K[88]);
    K[89] = Ops::fmac(vol, 0.006772486772486773, K[89]);
    K[90] = Ops::fmac(vol, -0.013544973544973546, K[90]);
    K[91] = Ops::fmac(vol, 0.006772486772486773, K[91]);
    K[92] = Ops::fmac(vol, 0.045149911816578486, K[92]);
    K[93] = Ops::fmac(vol, 0.009029982363315696, K[93]);
    K[94] = Ops::fmac(vol, -0.016931216931216932, K[94]);
    K[95] = Ops::fmac(vol, 0.022574955908289243, K[95]);
    K[96] = Ops::fmac(vol, 0.004514991181657848, K[96]);
    K[97] = Ops::fmac(vol, -0.004514991181657848, K[97]);
    K[98] = Ops::fmac(vol, 0.022574955908289243, K[98]);
    K[99] = Ops::fmac(vol, 0.045149911816578486, K[99]);
    K[100] = Ops::fmac(vol, -0.022574955908289243, K[100]);
    K[101] = Ops::fmac(vol, 0.013544973544973546, K[101]);
    K[102] = Ops::fmac(vol, -0.004514991181657848, K[102]);
    K[103] = Ops::fmac(vol, 0.022574955908289243, K[103]);
    K[104] = Ops::fmac(vol, 0.004514991181657848, K[104]);
    K[105] = Ops::fmac(vol, 0.05587301587301587, K[105]);
    K[106] = Ops::fmac(vol, -0.022574955908289243, K[106]);
    K[107] = Ops::fmac(vol, -0.013544973544973546, K[107]);
    K[108] = Ops::fmac(vol, 0.006772486772486773, K[108]);
    K[109] = Ops::fmac(vol, 0.006772486772486773, K[109]);
    K[110] = Ops::fmac(vol, 0.045149911816578486, K[110]);
    K[111] = Ops::fmac(vol, -0.004514991181657848, K[111]);
    K[112] = Ops::fmac(vol, 0.004514991181657848, K[112]);
    K[113] = Ops::fmac(vol, 0.022574955908289243, K[113]);
    K[114] = Ops::fmac(vol, 0.18962962962962962, K[114]);
    K[115] = Ops::fmac(vol, -0.02708994708994709, K[115]);
    K[116] = Ops::fmac(vol, -0.02708994708994709, K[116]);
    K[117] = Ops::fmac(vol, 0.18962962962962962, K[117]);
    K[118] = Ops::fmac(vol, -0.02708994708994709, K[118]);
    K[119] = Ops::fmac(vol, 0.18962962962962962, K[119]);
  }
  template <class Ops> __device__ __forceinline__ static void mass_upper(const typename Ops::T& vol, typename Ops::T* K) {
    K[0] = Ops::mulc(vol, 0.0051146384479717815);
    K[1] = Ops::mulc(vol, -0.0004761904761904762);
    K[2] = Ops::mulc(vol, -0.0004761904761904762);
    K[3] = Ops::mulc(vol, 0.0028218694885361554);
    K[4] = Ops::mulc(vol, -0.0014109347442680777);
    K[5] = Ops::mulc(vol, 0.0);
    K[6] = Ops::mulc(vol, 0.0028218694885361554);
    K[7] = Ops::mulc(vol, -0.0014109347442680777);
    K[8] = Ops::mulc(vol, 0.0);
    K[9] = Ops::mulc(vol, -0.0019753086419753087);
    K[10] = Ops::mulc(vol, -0.00021164021164021165);
    K[11] = Ops::mulc(vol, -0.0019753086419753087);
    K[12] = Ops::mulc(vol, 0.0028218694885361554);
    K[13] = Ops::mulc(vol, -0.0028218694885361554);
    K[14] = Ops::mulc(vol, -0.0028218694885361554);
    K[15] = Ops::mulc(vol, 0.0051146384479717815);
    K[16] = Ops::mulc(vol, -0.0004761904761904762);
    K[17] = Ops::mulc(vol, 0.0);
    K[18] = Ops::mulc(vol, -0.0014109347442680777);
    K[19] = Ops::mulc(vol, 0.0028218694885361554);
    K[20] = Ops::mulc(vol, -0.0019753086419753087);
    K[21] = Ops::mulc(vol, -0.00021164021164021165);
    K[22] = Ops::mulc(vol, -0.0019753086419753087);
    K[23] = Ops::mulc(vol, 0.0028218694885361554);
    K[24] = Ops::mulc(vol, -0.0014109347442680777);
    K[25] = Ops::mulc(vol, 0.0);
    K[26] = Ops::mulc(vol, -0.0028218694885361554);
    K[27] = Ops::mulc(vol, 0.0028218694885361554);
    K[28] = Ops::mulc(vol, -0.0028218694885361554);
    K[29] = Ops::mulc(vol, 0.0051146384479717815);
    K[30] = Ops::mulc(vol, -0.0019753086419753087);
    K[31] = Ops::mulc(vol, -0.00021164021164021165);
    K[32] = Ops::mulc(vol, -0.0019753086419753087);
    K[33] = Ops::mulc(vol, 0.0);
    K[34] = Ops::mulc(vol, -0.0014109347442680777);
    K[35] = Ops::mulc(vol, 0.0028218694885361554);
    K[36] = Ops::mulc(vol, 0.0);
    K[37] = Ops::mulc(vol, -0.0014109347442680777);
    K[38] = Ops::mulc(vol, 0.0028218694885361554);
    K[39] = Ops::mulc(vol, -0.0028218694885361554);
    K[40] = Ops::mulc(vol, -0.0028218694885361554);
    K[41] = Ops::mulc(vol, 0.0028218694885361554);
    K[42] = Ops::mulc(vol, 0.045149911816578486);
    K[43] = Ops::mulc(vol, -0.022574955908289243);
    K[44] = Ops::mulc(vol, 0.013544973544973546);
    K[45] = Ops::mulc(vol, 0.022574955908289243);
    K[46] = Ops::mulc(vol, -0.016931216931216932);
    K[47] = Ops::mulc(vol, 0.009029982363315696);
    K[48] = Ops::mulc(vol, 0.009029982363315696);
    K[49] = Ops::mulc(vol, 0.001128747795414462);
    K[50] = Ops::mulc(vol, 0.004514991181657848);
    K[51] = Ops::mulc(vol, 0.022574955908289243);
    K[52] = Ops::mulc(vol, 0.004514991181657848);
    K[53] = Ops::mulc(vol, -0.004514991181657848);
    K[54] = Ops::mulc(vol, 0.05587301587301587);
    K[55] = Ops::mulc(vol, -0.022574955908289243);
    K[56] = Ops::mulc(vol, -0.016931216931216932);
    K[57] = Ops::mulc(vol, 0.0008465608465608466);
    K[58] = Ops::mulc(vol, 0.001128747795414462);
    K[59] = Ops::mulc(vol, -0.016931216931216932);
    K[60] = Ops::mulc(vol, 0.0008465608465608466);
    K[61] = Ops::mulc(vol, 0.001128747795414462);
    K[62] = Ops::mulc(vol, 0.006772486772486773);
    K[63] = Ops::mulc(vol, 0.006772486772486773);
    K[64] = Ops::mulc(vol, -0.013544973544973546);
    K[65] = Ops::mulc(vol, 0.045149911816578486);
    K[66] = Ops::mulc(vol, 0.009029982363315696);
    K[67] = Ops::mulc(vol, 0.001128747795414462);
    K[68] = Ops::mulc(vol, 0.004514991181657848);
    K[69] = Ops::mulc(vol, 0.022574955908289243);
    K[70] = Ops::mulc(vol, -0.016931216931216932);
    K[71] = Ops::mulc(vol, 0.009029982363315696);
    K[72] = Ops::mulc(vol, 0.004514991181657848);
    K[73] = Ops::mulc(vol, 0.022574955908289243);
    K[74] = Ops::mulc(vol, -0.004514991181657848);
    K[75] = Ops::mulc(vol, 0.045149911816578486);
    K[76] = Ops::mulc(vol, -0.022574955908289243);
    K[77] = Ops::mulc(vol, 0.013544973544973546);
    K[78] = Ops::mulc(vol, 0.004514991181657848);
    K[79] = Ops::mulc(vol, 0.001128747795414462);
    K[80] = Ops::mulc(vol, 0.009029982363315696);
    K[81] = Ops::mulc(vol, 0.022574955908289243);
    K[82] = Ops::mulc(vol, -0.004514991181657848);
    K[83] = Ops::mulc(vol, 0.004514991181657848);
    K[84] = Ops::mulc(vol, 0.05587301587301587);
    K[85] = Ops::mulc(vol, -0.022574955908289243);
    K[86] = Ops::mulc(vol, 0.001128747795414462);
    K[87] = Ops::mulc(vol, 0.0008465608465608466);
    K[88] = Ops::mulc(vol, -0.016931216931216932);
    K[89] = Ops::mulc(vol, 0.006772486772486773);
    K[90] = Ops::mulc(vol, -0.013544973544973546);
    K[91] = Ops::mulc(vol, 0.006772486772486773);
    K[92] = Ops::mulc(vol, 0.045149911816578486);
    K[93] = Ops::mulc(vol, 0.009029982363315696);
    K[94] = Ops::mulc(vol, -0.016931216931216932);
    K[95] = Ops::mulc(vol, 0.022574955908289243);
    K[96] = Ops::mulc(vol, 0.004514991181657848);
    K[97] = Ops::mulc(vol, -0.004514991181657848);
    K[98] = Ops::mulc(vol, 0.022574955908289243);
    K[99] = Ops::mulc(vol, 0.045149911816578486);
    K[100] = Ops::mulc(vol, -0.022574955908289243);
    K[101] = Ops::mulc(vol, 0.013544973544973546);
    K[102] = Ops::mulc(vol, -0.004514991181657848);
    K[103] = Ops::mulc(vol, 0.022574955908289243);
    K[104] = Ops::mulc(vol, 0.004514991181657848);
    K[105] = Ops::mulc(vol, 0.05587301587301587);
    K[106] = Ops::mulc(vol, -0.022574955908289243);
    K[107] = Ops::mulc(vol, -0.013544973544973546);
    K[108] = Ops::mulc(vol, 0.006772486772486773);
    K[109] = Ops::mulc(vol, 0.006772486772486773);
    K[110] = Ops::mulc(vol, 0.045149911816578486);
    K[111] = Ops::mulc(vol, -0.004514991181657848);
    K[112] = Ops::mulc(vol, 0.004514991181657848);
    K[113] = Ops::mulc(vol, 0.022574955908289243);
    K[114] = Ops::mulc(vol, 0.18962962962962962);
    K[115] = Ops::mulc(vol, -0.02708994708994709);
    K[116] = Ops::mulc(vol, -0.02708994708994709);
    K[117] = Ops::mulc(vol, 0.18962962962962962);
    K[118] = Ops::mulc(vol, -0.02708994708994709);
    K[119] = Ops::mulc(vol, 0.18962962962962962);
  }
  template <class Ops, bool STIFF, bool MASS> __device__ __forceinline__ static void action_upper(const typename Ops::T* Lam, const typename Ops::T& vol, const typename Ops::T* x, typename Ops::T* y) {
    typename Ops::T k;
    { if constexpr (STIFF) { k = Ops::mulc(Lam[0], 0.746031746031746); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, 0.0051146384479717815, k); } y[0] = Ops::fma3(k, x[0], y[0]); }
    { if constexpr (STIFF) { k = Ops::mulc(Lam[1], -0.11322751322751323); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, -0.0004761904761904762, k); } y[0] = Ops::fma3(k, x[1], y[0]); y[1] = Ops::fma3(k, x[0], y[1]); }
    { if constexpr (STIFF) { k = Ops::mulc(Lam[2], -0.11322751322751323); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, -0.0004761904761904762, k); } y[0] = Ops::fma3(k, x[2], y[0]); y[2] = Ops::fma3(k, x[0], y[2]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[1], 1.5576719576719578, Ops::mulc(Lam[0], 0.25396825396825395)); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, 0.0028218694885361554, k); } y[0] = Ops::fma3(k, x[3], y[0]); y[3] = Ops::fma3(k, x[0], y[3]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[1], -0.8507936507936508, Ops::mulc(Lam[0], 0.08465608465608465)); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, -0.0014109347442680777, k); } y[0] = Ops::fma3(k, x[4], y[0]); y[4] = Ops::fma3(k, x[0], y[4]); }
    if constexpr (STIFF) { if constexpr (STIFF) { k = Ops::fmac(Lam[1], 0.40634920634920635, Ops::mulc(Lam[0], -0.08465608465608465)); } else { k = Ops::zero(); } y[0] = Ops::fma3(k, x[5], y[0]); y[5] = Ops::fma3(k, x[0], y[5]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[2], 1.5576719576719578, Ops::mulc(Lam[0], 0.25396825396825395)); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, 0.0028218694885361554, k); } y[0] = Ops::fma3(k, x[6], y[0]); y[6] = Ops::fma3(k, x[0], y[6]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[2], -0.8507936507936508, Ops::mulc(Lam[0], 0.08465608465608465)); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, -0.0014109347442680777, k); } y[0] = Ops::fma3(k, x[7], y[0]); y[7] = Ops::fma3(k, x[0], y[7]); }
    if constexpr (STIFF) { if constexpr (STIFF) { k = Ops::fmac(Lam[2], 0.40634920634920635, Ops::mulc(Lam[0], -0.08465608465608465)); } else { k = Ops::zero(); } y[0] = Ops::fma3(k, x[8], y[0]); y[8] = Ops::fma3(k, x[0], y[8]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[2], -0.08465608465608465, Ops::mulc(Lam[1], -0.08465608465608465)); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, -0.0019753086419753087, k); } y[0] = Ops::fma3(k, x[9], y[0]); y[9] = Ops::fma3(k, x[0], y[9]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[2], -0.08465608465608465, Ops::mulc(Lam[1], -0.08465608465608465)); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, -0.00021164021164021165, k); } y[0] = Ops::fma3(k, x[10], y[0]); y[10] = Ops::fma3(k, x[0], y[10]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[2], -0.08465608465608465, Ops::mulc(Lam[1], -0.08465608465608465)); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, -0.0019753086419753087, k); } y[0] = Ops::fma3(k, x[11], y[0]); y[11] = Ops::fma3(k, x[0], y[11]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[2], 0.6349206349206349, Ops::fmac(Lam[1], 0.6349206349206349, Ops::mulc(Lam[0], 0.4656084656084656))); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, 0.0028218694885361554, k); } y[0] = Ops::fma3(k, x[12], y[0]); y[12] = Ops::fma3(k, x[0], y[12]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[2], -0.042328042328042326, Ops::fmac(Lam[1], -0.042328042328042326, Ops::mulc(Lam[0], -0.21164021164021163))); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, -0.0028218694885361554, k); } y[0] = Ops::fma3(k, x[13], y[0]); y[13] = Ops::fma3(k, x[0], y[13]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[2], -0.042328042328042326, Ops::fmac(Lam[1], -0.042328042328042326, Ops::mulc(Lam[0], -0.21164021164021163))); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, -0.0028218694885361554, k); } y[0] = Ops::fma3(k, x[14], y[0]); y[14] = Ops::fma3(k, x[0], y[14]); }
    { if constexpr (STIFF) { k = Ops::mulc(Lam[3], 0.746031746031746); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, 0.0051146384479717815, k); } y[1] = Ops::fma3(k, x[1], y[1]); }
    { if constexpr (STIFF) { k = Ops::mulc(Lam[4], -0.11322751322751323); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, -0.0004761904761904762, k); } y[1] = Ops::fma3(k, x[2], y[1]); y[2] = Ops::fma3(k, x[1], y[2]); }
    if constexpr (STIFF) { if constexpr (STIFF) { k = Ops::fmac(Lam[3], -0.08465608465608465, Ops::mulc(Lam[1], 0.40634920634920635)); } else { k = Ops::zero(); } y[1] = Ops::fma3(k, x[3], y[1]); y[3] = Ops::fma3(k, x[1], y[3]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[3], 0.08465608465608465, Ops::mulc(Lam[1], -0.8507936507936508)); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, -0.0014109347442680777, k); } y[1] = Ops::fma3(k, x[4], y[1]); y[4] = Ops::fma3(k, x[1], y[4]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[3], 0.25396825396825395, Ops::mulc(Lam[1], 1.5576719576719578)); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, 0.0028218694885361554, k); } y[1] = Ops::fma3(k, x[5], y[1]); y[5] = Ops::fma3(k, x[1], y[5]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[4], -0.08465608465608465, Ops::mulc(Lam[1], -0.08465608465608465)); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, -0.0019753086419753087, k); } y[1] = Ops::fma3(k, x[6], y[1]); y[6] = Ops::fma3(k, x[1], y[6]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[4], -0.08465608465608465, Ops::mulc(Lam[1], -0.08465608465608465)); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, -0.00021164021164021165, k); } y[1] = Ops::fma3(k, x[7], y[1]); y[7] = Ops::fma3(k, x[1], y[7]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[4], -0.08465608465608465, Ops::mulc(Lam[1], -0.08465608465608465)); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, -0.0019753086419753087, k); } y[1] = Ops::fma3(k, x[8], y[1]); y[8] = Ops::fma3(k, x[1], y[8]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[4], 1.5576719576719578, Ops::mulc(Lam[3], 0.25396825396825395)); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, 0.0028218694885361554, k); } y[1] = Ops::fma3(k, x[9], y[1]); y[9] = Ops::fma3(k, x[1], y[9]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[4], -0.8507936507936508, Ops::mulc(Lam[3], 0.08465608465608465)); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, -0.0014109347442680777, k); } y[1] = Ops::fma3(k, x[10], y[1]); y[10] = Ops::fma3(k, x[1], y[10]); }
    if constexpr (STIFF) { if constexpr (STIFF) { k = Ops::fmac(Lam[4], 0.40634920634920635, Ops::mulc(Lam[3], -0.08465608465608465)); } else { k = Ops::zero(); } y[1] = Ops::fma3(k, x[11], y[1]); y[11] = Ops::fma3(k, x[1], y[11]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[4], -0.042328042328042326, Ops::fmac(Lam[3], -0.21164021164021163, Ops::mulc(Lam[1], -0.042328042328042326))); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, -0.0028218694885361554, k); } y[1] = Ops::fma3(k, x[12], y[1]); y[12] = Ops::fma3(k, x[1], y[12]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[4], 0.6349206349206349, Ops::fmac(Lam[3], 0.4656084656084656, Ops::mulc(Lam[1], 0.6349206349206349))); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, 0.0028218694885361554, k); } y[1] = Ops::fma3(k, x[13], y[1]); y[13] = Ops::fma3(k, x[1], y[13]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[4], -0.042328042328042326, Ops::fmac(Lam[3], -0.21164021164021163, Ops::mulc(Lam[1], -0.042328042328042326))); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, -0.0028218694885361554, k); } y[1] = Ops::fma3(k, x[14], y[1]); y[14] = Ops::fma3(k, x[1], y[14]); }
    { if constexpr (STIFF) { k = Ops::mulc(Lam[5], 0.746031746031746); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, 0.0051146384479717815, k); } y[2] = Ops::fma3(k, x[2], y[2]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[4], -0.08465608465608465, Ops::mulc(Lam[2], -0.08465608465608465)); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, -0.0019753086419753087, k); } y[2] = Ops::fma3(k, x[3], y[2]); y[3] = Ops::fma3(k, x[2], y[3]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[4], -0.08465608465608465, Ops::mulc(Lam[2], -0.08465608465608465)); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, -0.00021164021164021165, k); } y[2] = Ops::fma3(k, x[4], y[2]); y[4] = Ops::fma3(k, x[2], y[4]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[4], -0.08465608465608465, Ops::mulc(Lam[2], -0.08465608465608465)); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, -0.0019753086419753087, k); } y[2] = Ops::fma3(k, x[5], y[2]); y[5] = Ops::fma3(k, x[2], y[5]); }
    if constexpr (STIFF) { if constexpr (STIFF) { k = Ops::fmac(Lam[5], -0.08465608465608465, Ops::mulc(Lam[2], 0.40634920634920635)); } else { k = Ops::zero(); } y[2] = Ops::fma3(k, x[6], y[2]); y[6] = Ops::fma3(k, x[2], y[6]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[5], 0.08465608465608465, Ops::mulc(Lam[2], -0.8507936507936508)); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, -0.0014109347442680777, k); } y[2] = Ops::fma3(k, x[7], y[2]); y[7] = Ops::fma3(k, x[2], y[7]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[5], 0.25396825396825395, Ops::mulc(Lam[2], 1.5576719576719578)); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, 0.0028218694885361554, k); } y[2] = Ops::fma3(k, x[8], y[2]); y[8] = Ops::fma3(k, x[2], y[8]); }
    if constexpr (STIFF) { if constexpr (STIFF) { k = Ops::fmac(Lam[5], -0.08465608465608465, Ops::mulc(Lam[4], 0.40634920634920635)); } else { k = Ops::zero(); } y[2] = Ops::fma3(k, x[9], y[2]); y[9] = Ops::fma3(k, x[2], y[9]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[5], 0.08465608465608465, Ops::mulc(Lam[4], -0.8507936507936508)); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, -0.0014109347442680777, k); } y[2] = Ops::fma3(k, x[10], y[2]); y[10] = Ops::fma3(k, x[2], y[10]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[5], 0.25396825396825395, Ops::mulc(Lam[4], 1.5576719576719578)); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, 0.0028218694885361554, k); } y[2] = Ops::fma3(k, x[11], y[2]); y[11] = Ops::fma3(k, x[2], y[11]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[5], -0.21164021164021163, Ops::fmac(Lam[4], -0.042328042328042326, Ops::mulc(Lam[2], -0.042328042328042326))); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, -0.0028218694885361554, k); } y[2] = Ops::fma3(k, x[12], y[2]); y[12] = Ops::fma3(k, x[2], y[12]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[5], -0.21164021164021163, Ops::fmac(Lam[4], -0.042328042328042326, Ops::mulc(Lam[2], -0.042328042328042326))); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, -0.0028218694885361554, k); } y[2] = Ops::fma3(k, x[13], y[2]); y[13] = Ops::fma3(k, x[2], y[13]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[5], 0.4656084656084656, Ops::fmac(Lam[4], 0.6349206349206349, Ops::mulc(Lam[2], 0.6349206349206349))); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, 0.0028218694885361554, k); } y[2] = Ops::fma3(k, x[14], y[2]); y[14] = Ops::fma3(k, x[2], y[14]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[3], 4.1989417989417985, Ops::fmac(Lam[1], 4.1989417989417985, Ops::mulc(Lam[0], 3.657142857142857))); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, 0.045149911816578486, k); } y[3] = Ops::fma3(k, x[3], y[3]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[3], -1.5238095238095237, Ops::fmac(Lam[1], 1.0497354497354496, Ops::mulc(Lam[0], -1.3206349206349206))); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, -0.022574955908289243, k); } y[3] = Ops::fma3(k, x[4], y[3]); y[4] = Ops::fma3(k, x[3], y[4]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[3], 0.6772486772486772, Ops::fmac(Lam[1], -0.6772486772486772, Ops::mulc(Lam[0], 0.6772486772486772))); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, 0.013544973544973546, k); } y[3] = Ops::fma3(k, x[5], y[3]); y[5] = Ops::fma3(k, x[3], y[5]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[4], 4.1989417989417985, Ops::fmac(Lam[2], 2.0994708994708993, Ops::fmac(Lam[1], 2.0994708994708993, Ops::mulc(Lam[0], 1.8285714285714285)))); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, 0.022574955908289243, k); } y[3] = Ops::fma3(k, x[6], y[3]); y[6] = Ops::fma3(k, x[3], y[6]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[4], -1.5238095238095237, Ops::fmac(Lam[2], -0.9312169312169312, Ops::fmac(Lam[1], -0.5925925925925926, Ops::mulc(Lam[0], -0.728042328042328)))); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, -0.016931216931216932, k); } y[3] = Ops::fma3(k, x[7], y[3]); y[7] = Ops::fma3(k, x[3], y[7]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[4], 0.6772486772486772, Ops::fmac(Lam[2], 0.4740740740740741, Ops::fmac(Lam[1], 0.20317460317460317, Ops::mulc(Lam[0], 0.20317460317460317)))); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, 0.009029982363315696, k); } y[3] = Ops::fma3(k, x[8], y[3]); y[8] = Ops::fma3(k, x[3], y[8]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[4], 0.20317460317460317, Ops::fmac(Lam[3], 0.20317460317460317, Ops::fmac(Lam[2], 0.6772486772486772, Ops::mulc(Lam[1], 0.4740740740740741)))); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, 0.009029982363315696, k); } y[3] = Ops::fma3(k, x[9], y[3]); y[9] = Ops::fma3(k, x[3], y[9]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[4], 0.08465608465608465, Ops::fmac(Lam[3], 0.08465608465608465, Ops::fmac(Lam[2], 0.3047619047619048, Ops::mulc(Lam[1], 0.2201058201058201)))); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, 0.001128747795414462, k); } y[3] = Ops::fma3(k, x[10], y[3]); y[10] = Ops::fma3(k, x[3], y[10]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[4], 0.20317460317460317, Ops::fmac(Lam[3], 0.20317460317460317, Ops::fmac(Lam[2], 0.40634920634920635, Ops::mulc(Lam[1], 0.20317460317460317)))); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, 0.004514991181657848, k); } y[3] = Ops::fma3(k, x[11], y[3]); y[11] = Ops::fma3(k, x[3], y[11]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[4], 3.250793650793651, Ops::fmac(Lam[3], 3.250793650793651, Ops::fmac(Lam[2], 5.147089947089947, Ops::fmac(Lam[1], 3.250793650793651, Ops::mulc(Lam[0], 0.2708994708994709))))); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, 0.022574955908289243, k); } y[3] = Ops::fma3(k, x[12], y[3]); y[12] = Ops::fma3(k, x[3], y[12]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[4], -0.5417989417989418, Ops::fmac(Lam[3], -0.5417989417989418, Ops::fmac(Lam[2], -0.8126984126984127, Ops::mulc(Lam[0], 0.8126984126984127)))); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, 0.004514991181657848, k); } y[3] = Ops::fma3(k, x[13], y[3]); y[13] = Ops::fma3(k, x[3], y[13]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[4], -0.5417989417989418, Ops::fmac(Lam[3], -0.5417989417989418, Ops::fmac(Lam[2], -1.3544973544973544, Ops::fmac(Lam[1], -0.5417989417989418, Ops::mulc(Lam[0], 0.2708994708994709))))); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, -0.004514991181657848, k); } y[3] = Ops::fma3(k, x[14], y[3]); y[14] = Ops::fma3(k, x[3], y[14]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[3], 4.901587301587302, Ops::fmac(Lam[1], 3.8857142857142857, Ops::mulc(Lam[0], 4.901587301587302))); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, 0.05587301587301587, k); } y[4] = Ops::fma3(k, x[4], y[4]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[3], -1.3206349206349206, Ops::fmac(Lam[1], 1.0497354497354496, Ops::mulc(Lam[0], -1.5238095238095237))); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, -0.022574955908289243, k); } y[4] = Ops::fma3(k, x[5], y[4]); y[5] = Ops::fma3(k, x[4], y[5]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[4], -1.5238095238095237, Ops::fmac(Lam[2], -0.5925925925925926, Ops::fmac(Lam[1], -0.9312169312169312, Ops::mulc(Lam[0], -0.728042328042328)))); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, -0.016931216931216932, k); } y[4] = Ops::fma3(k, x[6], y[4]); y[6] = Ops::fma3(k, x[4], y[6]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[4], -0.7873015873015873, Ops::fmac(Lam[2], -0.39365079365079364, Ops::fmac(Lam[1], -0.39365079365079364, Ops::mulc(Lam[0], -0.2920634920634921)))); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, 0.0008465608465608466, k); } y[4] = Ops::fma3(k, x[7], y[4]); y[7] = Ops::fma3(k, x[4], y[7]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[4], 0.3047619047619048, Ops::fmac(Lam[2], 0.2201058201058201, Ops::fmac(Lam[1], 0.08465608465608465, Ops::mulc(Lam[0], 0.08465608465608465)))); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, 0.001128747795414462, k); } y[4] = Ops::fma3(k, x[8], y[4]); y[8] = Ops::fma3(k, x[4], y[8]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[4], -0.5925925925925926, Ops::fmac(Lam[3], -0.728042328042328, Ops::fmac(Lam[2], -1.5238095238095237, Ops::mulc(Lam[1], -0.9312169312169312)))); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, -0.016931216931216932, k); } y[4] = Ops::fma3(k, x[9], y[4]); y[9] = Ops::fma3(k, x[4], y[9]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[4], -0.39365079365079364, Ops::fmac(Lam[3], -0.2920634920634921, Ops::fmac(Lam[2], -0.7873015873015873, Ops::mulc(Lam[1], -0.39365079365079364)))); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, 0.0008465608465608466, k); } y[4] = Ops::fma3(k, x[10], y[4]); y[10] = Ops::fma3(k, x[4], y[10]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[4], 0.2201058201058201, Ops::fmac(Lam[3], 0.08465608465608465, Ops::fmac(Lam[2], 0.3047619047619048, Ops::mulc(Lam[1], 0.08465608465608465)))); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, 0.001128747795414462, k); } y[4] = Ops::fma3(k, x[11], y[4]); y[11] = Ops::fma3(k, x[4], y[11]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[4], 4.673015873015873, Ops::fmac(Lam[3], -1.0158730158730158, Ops::fmac(Lam[2], 1.8285714285714285, Ops::fmac(Lam[1], 1.8285714285714285, Ops::mulc(Lam[0], 2.641269841269841))))); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, 0.006772486772486773, k); } y[4] = Ops::fma3(k, x[12], y[4]); y[12] = Ops::fma3(k, x[4], y[12]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[4], 1.8285714285714285, Ops::fmac(Lam[3], 2.641269841269841, Ops::fmac(Lam[2], 4.673015873015873, Ops::fmac(Lam[1], 1.8285714285714285, Ops::mulc(Lam[0], -1.0158730158730158))))); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, 0.006772486772486773, k); } y[4] = Ops::fma3(k, x[13], y[4]); y[13] = Ops::fma3(k, x[4], y[13]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[4], -1.4222222222222223, Ops::fmac(Lam[3], -0.6095238095238096, Ops::fmac(Lam[2], -1.4222222222222223, Ops::fmac(Lam[1], -1.0158730158730158, Ops::mulc(Lam[0], -0.6095238095238096))))); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, -0.013544973544973546, k); } y[4] = Ops::fma3(k, x[14], y[4]); y[14] = Ops::fma3(k, x[4], y[14]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[3], 3.657142857142857, Ops::fmac(Lam[1], 4.1989417989417985, Ops::mulc(Lam[0], 4.1989417989417985))); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, 0.045149911816578486, k); } y[5] = Ops::fma3(k, x[5], y[5]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[4], 0.6772486772486772, Ops::fmac(Lam[2], 0.20317460317460317, Ops::fmac(Lam[1], 0.4740740740740741, Ops::mulc(Lam[0], 0.20317460317460317)))); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, 0.009029982363315696, k); } y[5] = Ops::fma3(k, x[6], y[5]); y[6] = Ops::fma3(k, x[5], y[6]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[4], 0.3047619047619048, Ops::fmac(Lam[2], 0.08465608465608465, Ops::fmac(Lam[1], 0.2201058201058201, Ops::mulc(Lam[0], 0.08465608465608465)))); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, 0.001128747795414462, k); } y[5] = Ops::fma3(k, x[7], y[5]); y[7] = Ops::fma3(k, x[5], y[7]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[4], 0.40634920634920635, Ops::fmac(Lam[2], 0.20317460317460317, Ops::fmac(Lam[1], 0.20317460317460317, Ops::mulc(Lam[0], 0.20317460317460317)))); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, 0.004514991181657848, k); } y[5] = Ops::fma3(k, x[8], y[5]); y[8] = Ops::fma3(k, x[5], y[8]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[4], 2.0994708994708993, Ops::fmac(Lam[3], 1.8285714285714285, Ops::fmac(Lam[2], 4.1989417989417985, Ops::mulc(Lam[1], 2.0994708994708993)))); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, 0.022574955908289243, k); } y[5] = Ops::fma3(k, x[9], y[5]); y[9] = Ops::fma3(k, x[5], y[9]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[4], -0.9312169312169312, Ops::fmac(Lam[3], -0.728042328042328, Ops::fmac(Lam[2], -1.5238095238095237, Ops::mulc(Lam[1], -0.5925925925925926)))); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, -0.016931216931216932, k); } y[5] = Ops::fma3(k, x[10], y[5]); y[10] = Ops::fma3(k, x[5], y[10]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[4], 0.4740740740740741, Ops::fmac(Lam[3], 0.20317460317460317, Ops::fmac(Lam[2], 0.6772486772486772, Ops::mulc(Lam[1], 0.20317460317460317)))); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, 0.009029982363315696, k); } y[5] = Ops::fma3(k, x[11], y[5]); y[11] = Ops::fma3(k, x[5], y[11]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[4], -0.8126984126984127, Ops::fmac(Lam[3], 0.8126984126984127, Ops::fmac(Lam[2], -0.5417989417989418, Ops::mulc(Lam[0], -0.5417989417989418)))); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, 0.004514991181657848, k); } y[5] = Ops::fma3(k, x[12], y[5]); y[12] = Ops::fma3(k, x[5], y[12]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[4], 5.147089947089947, Ops::fmac(Lam[3], 0.2708994708994709, Ops::fmac(Lam[2], 3.250793650793651, Ops::fmac(Lam[1], 3.250793650793651, Ops::mulc(Lam[0], 3.250793650793651))))); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, 0.022574955908289243, k); } y[5] = Ops::fma3(k, x[13], y[5]); y[13] = Ops::fma3(k, x[5], y[13]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[4], -1.3544973544973544, Ops::fmac(Lam[3], 0.2708994708994709, Ops::fmac(Lam[2], -0.5417989417989418, Ops::fmac(Lam[1], -0.5417989417989418, Ops::mulc(Lam[0], -0.5417989417989418))))); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, -0.004514991181657848, k); } y[5] = Ops::fma3(k, x[14], y[5]); y[14] = Ops::fma3(k, x[5], y[14]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[5], 4.1989417989417985, Ops::fmac(Lam[2], 4.1989417989417985, Ops::mulc(Lam[0], 3.657142857142857))); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, 0.045149911816578486, k); } y[6] = Ops::fma3(k, x[6], y[6]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[5], -1.5238095238095237, Ops::fmac(Lam[2], 1.0497354497354496, Ops::mulc(Lam[0], -1.3206349206349206))); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, -0.022574955908289243, k); } y[6] = Ops::fma3(k, x[7], y[6]); y[7] = Ops::fma3(k, x[6], y[7]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[5], 0.6772486772486772, Ops::fmac(Lam[2], -0.6772486772486772, Ops::mulc(Lam[0], 0.6772486772486772))); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, 0.013544973544973546, k); } y[6] = Ops::fma3(k, x[8], y[6]); y[8] = Ops::fma3(k, x[6], y[8]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[5], 0.20317460317460317, Ops::fmac(Lam[4], 0.20317460317460317, Ops::fmac(Lam[2], 0.20317460317460317, Ops::mulc(Lam[1], 0.40634920634920635)))); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, 0.004514991181657848, k); } y[6] = Ops::fma3(k, x[9], y[6]); y[9] = Ops::fma3(k, x[6], y[9]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[5], 0.08465608465608465, Ops::fmac(Lam[4], 0.08465608465608465, Ops::fmac(Lam[2], 0.2201058201058201, Ops::mulc(Lam[1], 0.3047619047619048)))); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, 0.001128747795414462, k); } y[6] = Ops::fma3(k, x[10], y[6]); y[10] = Ops::fma3(k, x[6], y[10]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[5], 0.20317460317460317, Ops::fmac(Lam[4], 0.20317460317460317, Ops::fmac(Lam[2], 0.4740740740740741, Ops::mulc(Lam[1], 0.6772486772486772)))); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, 0.009029982363315696, k); } y[6] = Ops::fma3(k, x[11], y[6]); y[11] = Ops::fma3(k, x[6], y[11]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[5], 3.250793650793651, Ops::fmac(Lam[4], 3.250793650793651, Ops::fmac(Lam[2], 3.250793650793651, Ops::fmac(Lam[1], 5.147089947089947, Ops::mulc(Lam[0], 0.2708994708994709))))); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, 0.022574955908289243, k); } y[6] = Ops::fma3(k, x[12], y[6]); y[12] = Ops::fma3(k, x[6], y[12]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[5], -0.5417989417989418, Ops::fmac(Lam[4], -0.5417989417989418, Ops::fmac(Lam[2], -0.5417989417989418, Ops::fmac(Lam[1], -1.3544973544973544, Ops::mulc(Lam[0], 0.2708994708994709))))); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, -0.004514991181657848, k); } y[6] = Ops::fma3(k, x[13], y[6]); y[13] = Ops::fma3(k, x[6], y[13]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[5], -0.5417989417989418, Ops::fmac(Lam[4], -0.5417989417989418, Ops::fmac(Lam[1], -0.8126984126984127, Ops::mulc(Lam[0], 0.8126984126984127)))); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, 0.004514991181657848, k); } y[6] = Ops::fma3(k, x[14], y[6]); y[14] = Ops::fma3(k, x[6], y[14]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[5], 4.901587301587302, Ops::fmac(Lam[2], 3.8857142857142857, Ops::mulc(Lam[0], 4.901587301587302))); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, 0.05587301587301587, k); } y[7] = Ops::fma3(k, x[7], y[7]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[5], -1.3206349206349206, Ops::fmac(Lam[2], 1.0497354497354496, Ops::mulc(Lam[0], -1.5238095238095237))); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, -0.022574955908289243, k); } y[7] = Ops::fma3(k, x[8], y[7]); y[8] = Ops::fma3(k, x[7], y[8]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[5], 0.08465608465608465, Ops::fmac(Lam[4], 0.2201058201058201, Ops::fmac(Lam[2], 0.08465608465608465, Ops::mulc(Lam[1], 0.3047619047619048)))); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, 0.001128747795414462, k); } y[7] = Ops::fma3(k, x[9], y[7]); y[9] = Ops::fma3(k, x[7], y[9]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[5], -0.2920634920634921, Ops::fmac(Lam[4], -0.39365079365079364, Ops::fmac(Lam[2], -0.39365079365079364, Ops::mulc(Lam[1], -0.7873015873015873)))); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, 0.0008465608465608466, k); } y[7] = Ops::fma3(k, x[10], y[7]); y[10] = Ops::fma3(k, x[7], y[10]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[5], -0.728042328042328, Ops::fmac(Lam[4], -0.5925925925925926, Ops::fmac(Lam[2], -0.9312169312169312, Ops::mulc(Lam[1], -1.5238095238095237)))); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, -0.016931216931216932, k); } y[7] = Ops::fma3(k, x[11], y[7]); y[11] = Ops::fma3(k, x[7], y[11]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[5], -1.0158730158730158, Ops::fmac(Lam[4], 4.673015873015873, Ops::fmac(Lam[2], 1.8285714285714285, Ops::fmac(Lam[1], 1.8285714285714285, Ops::mulc(Lam[0], 2.641269841269841))))); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, 0.006772486772486773, k); } y[7] = Ops::fma3(k, x[12], y[7]); y[12] = Ops::fma3(k, x[7], y[12]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[5], -0.6095238095238096, Ops::fmac(Lam[4], -1.4222222222222223, Ops::fmac(Lam[2], -1.0158730158730158, Ops::fmac(Lam[1], -1.4222222222222223, Ops::mulc(Lam[0], -0.6095238095238096))))); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, -0.013544973544973546, k); } y[7] = Ops::fma3(k, x[13], y[7]); y[13] = Ops::fma3(k, x[7], y[13]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[5], 2.641269841269841, Ops::fmac(Lam[4], 1.8285714285714285, Ops::fmac(Lam[2], 1.8285714285714285, Ops::fmac(Lam[1], 4.673015873015873, Ops::mulc(Lam[0], -1.0158730158730158))))); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, 0.006772486772486773, k); } y[7] = Ops::fma3(k, x[14], y[7]); y[14] = Ops::fma3(k, x[7], y[14]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[5], 3.657142857142857, Ops::fmac(Lam[2], 4.1989417989417985, Ops::mulc(Lam[0], 4.1989417989417985))); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, 0.045149911816578486, k); } y[8] = Ops::fma3(k, x[8], y[8]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[5], 0.20317460317460317, Ops::fmac(Lam[4], 0.4740740740740741, Ops::fmac(Lam[2], 0.20317460317460317, Ops::mulc(Lam[1], 0.6772486772486772)))); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, 0.009029982363315696, k); } y[8] = Ops::fma3(k, x[9], y[8]); y[9] = Ops::fma3(k, x[8], y[9]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[5], -0.728042328042328, Ops::fmac(Lam[4], -0.9312169312169312, Ops::fmac(Lam[2], -0.5925925925925926, Ops::mulc(Lam[1], -1.5238095238095237)))); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, -0.016931216931216932, k); } y[8] = Ops::fma3(k, x[10], y[8]); y[10] = Ops::fma3(k, x[8], y[10]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[5], 1.8285714285714285, Ops::fmac(Lam[4], 2.0994708994708993, Ops::fmac(Lam[2], 2.0994708994708993, Ops::mulc(Lam[1], 4.1989417989417985)))); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, 0.022574955908289243, k); } y[8] = Ops::fma3(k, x[11], y[8]); y[11] = Ops::fma3(k, x[8], y[11]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[5], 0.8126984126984127, Ops::fmac(Lam[4], -0.8126984126984127, Ops::fmac(Lam[1], -0.5417989417989418, Ops::mulc(Lam[0], -0.5417989417989418)))); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, 0.004514991181657848, k); } y[8] = Ops::fma3(k, x[12], y[8]); y[12] = Ops::fma3(k, x[8], y[12]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[5], 0.2708994708994709, Ops::fmac(Lam[4], -1.3544973544973544, Ops::fmac(Lam[2], -0.5417989417989418, Ops::fmac(Lam[1], -0.5417989417989418, Ops::mulc(Lam[0], -0.5417989417989418))))); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, -0.004514991181657848, k); } y[8] = Ops::fma3(k, x[13], y[8]); y[13] = Ops::fma3(k, x[8], y[13]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[5], 0.2708994708994709, Ops::fmac(Lam[4], 5.147089947089947, Ops::fmac(Lam[2], 3.250793650793651, Ops::fmac(Lam[1], 3.250793650793651, Ops::mulc(Lam[0], 3.250793650793651))))); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, 0.022574955908289243, k); } y[8] = Ops::fma3(k, x[14], y[8]); y[14] = Ops::fma3(k, x[8], y[14]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[5], 4.1989417989417985, Ops::fmac(Lam[4], 4.1989417989417985, Ops::mulc(Lam[3], 3.657142857142857))); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, 0.045149911816578486, k); } y[9] = Ops::fma3(k, x[9], y[9]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[5], -1.5238095238095237, Ops::fmac(Lam[4], 1.0497354497354496, Ops::mulc(Lam[3], -1.3206349206349206))); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, -0.022574955908289243, k); } y[9] = Ops::fma3(k, x[10], y[9]); y[10] = Ops::fma3(k, x[9], y[10]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[5], 0.6772486772486772, Ops::fmac(Lam[4], -0.6772486772486772, Ops::mulc(Lam[3], 0.6772486772486772))); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, 0.013544973544973546, k); } y[9] = Ops::fma3(k, x[11], y[9]); y[11] = Ops::fma3(k, x[9], y[11]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[5], -0.5417989417989418, Ops::fmac(Lam[4], -0.5417989417989418, Ops::fmac(Lam[3], 0.2708994708994709, Ops::fmac(Lam[2], -0.5417989417989418, Ops::mulc(Lam[1], -1.3544973544973544))))); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, -0.004514991181657848, k); } y[9] = Ops::fma3(k, x[12], y[9]); y[12] = Ops::fma3(k, x[9], y[12]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[5], 3.250793650793651, Ops::fmac(Lam[4], 3.250793650793651, Ops::fmac(Lam[3], 0.2708994708994709, Ops::fmac(Lam[2], 3.250793650793651, Ops::mulc(Lam[1], 5.147089947089947))))); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, 0.022574955908289243, k); } y[9] = Ops::fma3(k, x[13], y[9]); y[13] = Ops::fma3(k, x[9], y[13]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[5], -0.5417989417989418, Ops::fmac(Lam[3], 0.8126984126984127, Ops::fmac(Lam[2], -0.5417989417989418, Ops::mulc(Lam[1], -0.8126984126984127)))); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, 0.004514991181657848, k); } y[9] = Ops::fma3(k, x[14], y[9]); y[14] = Ops::fma3(k, x[9], y[14]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[5], 4.901587301587302, Ops::fmac(Lam[4], 3.8857142857142857, Ops::mulc(Lam[3], 4.901587301587302))); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, 0.05587301587301587, k); } y[10] = Ops::fma3(k, x[10], y[10]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[5], -1.3206349206349206, Ops::fmac(Lam[4], 1.0497354497354496, Ops::mulc(Lam[3], -1.5238095238095237))); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, -0.022574955908289243, k); } y[10] = Ops::fma3(k, x[11], y[10]); y[11] = Ops::fma3(k, x[10], y[11]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[5], -0.6095238095238096, Ops::fmac(Lam[4], -1.0158730158730158, Ops::fmac(Lam[3], -0.6095238095238096, Ops::fmac(Lam[2], -1.4222222222222223, Ops::mulc(Lam[1], -1.4222222222222223))))); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, -0.013544973544973546, k); } y[10] = Ops::fma3(k, x[12], y[10]); y[12] = Ops::fma3(k, x[10], y[12]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[5], -1.0158730158730158, Ops::fmac(Lam[4], 1.8285714285714285, Ops::fmac(Lam[3], 2.641269841269841, Ops::fmac(Lam[2], 4.673015873015873, Ops::mulc(Lam[1], 1.8285714285714285))))); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, 0.006772486772486773, k); } y[10] = Ops::fma3(k, x[13], y[10]); y[13] = Ops::fma3(k, x[10], y[13]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[5], 2.641269841269841, Ops::fmac(Lam[4], 1.8285714285714285, Ops::fmac(Lam[3], -1.0158730158730158, Ops::fmac(Lam[2], 1.8285714285714285, Ops::mulc(Lam[1], 4.673015873015873))))); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, 0.006772486772486773, k); } y[10] = Ops::fma3(k, x[14], y[10]); y[14] = Ops::fma3(k, x[10], y[14]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[5], 3.657142857142857, Ops::fmac(Lam[4], 4.1989417989417985, Ops::mulc(Lam[3], 4.1989417989417985))); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, 0.045149911816578486, k); } y[11] = Ops::fma3(k, x[11], y[11]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[5], 0.2708994708994709, Ops::fmac(Lam[4], -0.5417989417989418, Ops::fmac(Lam[3], -0.5417989417989418, Ops::fmac(Lam[2], -1.3544973544973544, Ops::mulc(Lam[1], -0.5417989417989418))))); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, -0.004514991181657848, k); } y[11] = Ops::fma3(k, x[12], y[11]); y[12] = Ops::fma3(k, x[11], y[12]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[5], 0.8126984126984127, Ops::fmac(Lam[3], -0.5417989417989418, Ops::fmac(Lam[2], -0.8126984126984127, Ops::mulc(Lam[1], -0.5417989417989418)))); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, 0.004514991181657848, k); } y[11] = Ops::fma3(k, x[13], y[11]); y[13] = Ops::fma3(k, x[11], y[13]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[5], 0.2708994708994709, Ops::fmac(Lam[4], 3.250793650793651, Ops::fmac(Lam[3], 3.250793650793651, Ops::fmac(Lam[2], 5.147089947089947, Ops::mulc(Lam[1], 3.250793650793651))))); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, 0.022574955908289243, k); } y[11] = Ops::fma3(k, x[14], y[11]); y[14] = Ops::fma3(k, x[11], y[14]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[5], 11.377777777777778, Ops::fmac(Lam[4], 11.377777777777778, Ops::fmac(Lam[3], 11.377777777777778, Ops::fmac(Lam[2], 11.377777777777778, Ops::fmac(Lam[1], 11.377777777777778, Ops::mulc(Lam[0], 11.377777777777778)))))); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, 0.18962962962962962, k); } y[12] = Ops::fma3(k, x[12], y[12]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[5], 1.6253968253968254, Ops::fmac(Lam[4], 1.6253968253968254, Ops::fmac(Lam[3], -1.6253968253968254, Ops::fmac(Lam[2], 1.6253968253968254, Ops::fmac(Lam[1], 4.876190476190477, Ops::mulc(Lam[0], -1.6253968253968254)))))); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, -0.02708994708994709, k); } y[12] = Ops::fma3(k, x[13], y[12]); y[13] = Ops::fma3(k, x[12], y[13]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[5], -1.6253968253968254, Ops::fmac(Lam[4], 1.6253968253968254, Ops::fmac(Lam[3], 1.6253968253968254, Ops::fmac(Lam[2], 4.876190476190477, Ops::fmac(Lam[1], 1.6253968253968254, Ops::mulc(Lam[0], -1.6253968253968254)))))); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, -0.02708994708994709, k); } y[12] = Ops::fma3(k, x[14], y[12]); y[14] = Ops::fma3(k, x[12], y[14]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[5], 11.377777777777778, Ops::fmac(Lam[4], 11.377777777777778, Ops::fmac(Lam[3], 11.377777777777778, Ops::fmac(Lam[2], 11.377777777777778, Ops::fmac(Lam[1], 11.377777777777778, Ops::mulc(Lam[0], 11.377777777777778)))))); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, 0.18962962962962962, k); } y[13] = Ops::fma3(k, x[13], y[13]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[5], -1.6253968253968254, Ops::fmac(Lam[4], 4.876190476190477, Ops::fmac(Lam[3], -1.6253968253968254, Ops::fmac(Lam[2], 1.6253968253968254, Ops::fmac(Lam[1], 1.6253968253968254, Ops::mulc(Lam[0], 1.6253968253968254)))))); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, -0.02708994708994709, k); } y[13] = Ops::fma3(k, x[14], y[13]); y[14] = Ops::fma3(k, x[13], y[14]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[5], 11.377777777777778, Ops::fmac(Lam[4], 11.377777777777778, Ops::fmac(Lam[3], 11.377777777777778, Ops::fmac(Lam[2], 11.377777777777778, Ops::fmac(Lam[1], 11.377777777777778, Ops::mulc(Lam[0], 11.377777777777778)))))); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, 0.18962962962962962, k); } y[14] = Ops::fma3(k, x[14], y[14]); }
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
  template <class Ops> __device__ __forceinline__ static void mass_upper_add(const typename Ops::T& vol, typename Ops::T* K) {
    K[0] = Ops::fmac(vol, 0.1, K[0]);
    K[1] = Ops::fmac(vol, 0.05, K[1]);
    K[2] = Ops::fmac(vol, 0.05, K[2]);
    K[3] = Ops::fmac(vol, 0.05, K[3]);
    K[4] = Ops::fmac(vol, 0.1, K[4]);
    K[5] = Ops::fmac(vol, 0.05, K[5]);
    K[6] = Ops::fmac(vol, 0.05, K[6]);
    K[7] = Ops::fmac(vol, 0.1, K[7]);
    K[8] = Ops::fmac(vol, 0.05, K[8]);
    K[9] = Ops::fmac(vol, 0.1, K[9]);
  }
  template <class Ops> __device__ __forceinline__ static void mass_upper(const typename Ops::T& vol, typename Ops::T* K) {
    K[0] = Ops::mulc(vol, 0.1);
    K[1] = Ops::mulc(vol, 0.05);
    K[2] = Ops::mulc(vol, 0.05);
    K[3] = Ops::mulc(vol, 0.05);
    K[4] = Ops::mulc(vol, 0.1);
    K[5] = Ops::mulc(vol, 0.05);
    K[6] = Ops::mulc(vol, 0.05);
    K[7] = Ops::mulc(vol, 0.1);
    K[8] = Ops::mulc(vol, 0.05);
    K[9] = Ops::mulc(vol, 0.1);
  }
  template <class Ops, bool STIFF, bool MASS> __device__ __forceinline__ static void action_upper(const typename Ops::T* Lam, const typename Ops::T& vol, const typename Ops::T* x, typename Ops::T* y) {
    typename Ops::T k;
    { if constexpr (STIFF) { k = Lam[0]; } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, 0.1, k); } y[0] = Ops::fma3(k, x[0], y[0]); }
    { if constexpr (STIFF) { k = Lam[1]; } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, 0.05, k); } y[0] = Ops::fma3(k, x[1], y[0]); y[1] = Ops::fma3(k, x[0], y[1]); }
    { if constexpr (STIFF) { k = Lam[2]; } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, 0.05, k); } y[0] = Ops::fma3(k, x[2], y[0]); y[2] = Ops::fma3(k, x[0], y[2]); }
    { if constexpr (STIFF) { k = Lam[3]; } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, 0.05, k); } y[0] = Ops::fma3(k, x[3], y[0]); y[3] = Ops::fma3(k, x[0], y[3]); }
    { if constexpr (STIFF) { k = Lam[4]; } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, 0.1, k); } y[1] = Ops::fma3(k, x[1], y[1]); }
    { if constexpr (STIFF) { k = Lam[5]; } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, 0.05, k); } y[1] = Ops::fma3(k, x[2], y[1]); y[2] = Ops::fma3(k, x[1], y[2]); }
    { if constexpr (STIFF) { k = Lam[6]; } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, 0.05, k); } y[1] = Ops::fma3(k, x[3], y[1]); y[3] = Ops::fma3(k, x[1], y[3]); }
    { if constexpr (STIFF) { k = Lam[7]; } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, 0.1, k); } y[2] = Ops::fma3(k, x[2], y[2]); }
    { if constexpr (STIFF) { k = Lam[8]; } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, 0.05, k); } y[2] = Ops::fma3(k, x[3], y[2]); y[3] = Ops::fma3(k, x[2], y[3]); }
    { if constexpr (STIFF) { k = Lam[9]; } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, 0.1, k); } y[3] = Ops::fma3(k, x[3], y[3]); }
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
  template <class Ops> __device__ __forceinline__ static void stiffness_upper(const typename Ops::T* Lam, typename Ops::T* K) {
    K[0] = Ops::mulc(Lam[0], 0.6);
    K[1] = Ops::mulc(Lam[1], -0.2);
    K[2] = Ops::mulc(Lam[2], -0.2);
    K[3] = Ops::mulc(Lam[3], -0.2);
    K[4] = Ops::fmac(Lam[1], 0.6, Ops::mulc(Lam[0], -0.2));
    K[5] = Ops::fmac(Lam[2], 0.6, Ops::mulc(Lam[0], -0.2));
    K[6] = Ops::fmac(Lam[3], 0.6, Ops::mulc(Lam[0], -0.2));
    K[7] = Ops::fmac(Lam[2], -0.2, Ops::mulc(Lam[1], -0.2));
    K[8] = Ops::fmac(Lam[3], -0.2, Ops::mulc(Lam[1], -0.2));
    K[9] = Ops::fmac(Lam[3], -0.2, Ops::mulc(Lam[2], -0.2));
    K[10] = Ops::mulc(Lam[4], 0.6);
    K[11] = Ops::mulc(Lam[5], -0.2);
    K[12] = Ops::mulc(Lam[6], -0.2);
    K[13] = Ops::fmac(Lam[4], -0.2, Ops::mulc(Lam[1], 0.6));
    K[14] = Ops::fmac(Lam[5], -0.2, Ops::mulc(Lam[1], -0.2));
    K[15] = Ops::fmac(Lam[6], -0.2, Ops::mulc(Lam[1], -0.2));
    K[16] = Ops::fmac(Lam[5], 0.6, Ops::mulc(Lam[4], -0.2));
    K[17] = Ops::fmac(Lam[6], 0.6, Ops::mulc(Lam[4], -0.2));
    K[18] = Ops::fmac(Lam[6], -0.2, Ops::mulc(Lam[5], -0.2));
    K[19] = Ops::mulc(Lam[7], 0.6);
    K[20] = Ops::mulc(Lam[8], -0.2);
    K[21] = Ops::fmac(Lam[5], -0.2, Ops::mulc(Lam[2], -0.2));
    K[22] = Ops::fmac(Lam[7], -0.2, Ops::mulc(Lam[2], 0.6));
    K[23] = Ops::fmac(Lam[8], -0.2, Ops::mulc(Lam[2], -0.2));
    K[24] = Ops::fmac(Lam[7], -0.2, Ops::mulc(Lam[5], 0.6));
    K[25] = Ops::fmac(Lam[8], -0.2, Ops::mulc(Lam[5], -0.2));
    K[26] = Ops::fmac(Lam[8], 0.6, Ops::mulc(Lam[7], -0.2));
    K[27] = Ops::mulc(Lam[9], 0.6);
    K[28] = Ops::fmac(Lam[6], -0.2, Ops::mulc(Lam[3], -0.2));
    K[29] = Ops::fmac(Lam[8], -0.2, Ops::mulc(Lam[3], -0.2));
    K[30] = Ops::fmac(Lam[9], -0.2, Ops::mulc(Lam[3], 0.6));
    K[31] = Ops::fmac(Lam[8], -0.2, Ops::mulc(Lam[6], -0.2));
    K[32] = Ops::fmac(Lam[9], -0.2, Ops::mulc(Lam[6], 0.6));
    K[33] = Ops::fmac(Lam[9], -0.2, Ops::mulc(Lam[8], 0.6));
    K[34] = Ops::fmac(Lam[4], 1.6, Ops::fmac(Lam[1], 1.6, Ops::mulc(Lam[0], 1.6)));
    K[35] = Ops::fmac(Lam[5], 1.6, Ops::fmac(Lam[2], 0.8, Ops::fmac(Lam[1], 0.8, Ops::mulc(Lam[0], 0.8))));
    K[36] = Ops::fmac(Lam[6], 1.6, Ops::fmac(Lam[3], 0.8, Ops::fmac(Lam[1], 0.8, Ops::mulc(Lam[0], 0.8))));
    K[37] = Ops::fmac(Lam[5], 0.8, Ops::fmac(Lam[4], 0.8, Ops::fmac(Lam[2], 1.6, Ops::mulc(Lam[1], 0.8))));
    K[38] = Ops::fmac(Lam[6], 0.8, Ops::fmac(Lam[4], 0.8, Ops::fmac(Lam[3], 1.6, Ops::mulc(Lam[1], 0.8))));
    K[39] = Ops::fmac(Lam[6], 0.8, Ops::fmac(Lam[5], 0.8, Ops::fmac(Lam[3], 0.8, Ops::mulc(Lam[2], 0.8))));
    K[40] = Ops::fmac(Lam[7], 1.6, Ops::fmac(Lam[2], 1.6, Ops::mulc(Lam[0], 1.6)));
    K[41] = Ops::fmac(Lam[8], 1.6, Ops::fmac(Lam[3], 0.8, Ops::fmac(Lam[2], 0.8, Ops::mulc(Lam[0], 0.8))));
    K[42] = Ops::fmac(Lam[7], 0.8, Ops::fmac(Lam[5], 0.8, Ops::fmac(Lam[2], 0.8, Ops::mulc(Lam[1], 1.6))));
    K[43] = Ops::fmac(Lam[8], 0.8, Ops::fmac(Lam[5], 0.8, Ops::fmac(Lam[3], 0.8, Ops::mulc(Lam[1], 0.8))));
    K[44] = Ops::fmac(Lam[8], 0.8, Ops::fmac(Lam[7], 0.8, Ops::fmac(Lam[3], 1.6, Ops::mulc(Lam[2], 0.8))));
    K[45] = Ops::fmac(Lam[9], 1.6, Ops::fmac(Lam[3], 1.6, Ops::mulc(Lam[0], 1.6)));
    K[46] = Ops::fmac(Lam[8], 0.8, Ops::fmac(Lam[6], 0.8, Ops::fmac(Lam[2], 0.8, Ops::mulc(Lam[1], 0.8))));
    K[47] = Ops::fmac(Lam[9], 0.8, Ops::fmac(Lam[6], 0.8, Ops::fmac(Lam[3], 0.8, Ops::mulc(Lam[1], 1.6))));
    K[48] = Ops::fmac(Lam[9], 0.8, Ops::fmac(Lam[8], 0.8, Ops::fmac(Lam[3], 0.8, Ops::mulc(Lam[2], 1.6))));
    K[49] = Ops::fmac(Lam[7], 1.6, Ops::fmac(Lam[5], 1.6, Ops::mulc(Lam[4], 1.6)));
    K[50] = Ops::fmac(Lam[8], 1.6, Ops::fmac(Lam[6], 0.8, Ops::fmac(Lam[5], 0.8, Ops::mulc(Lam[4], 0.8))));
    K[51] = Ops::fmac(Lam[8], 0.8, Ops::fmac(Lam[7], 0.8, Ops::fmac(Lam[6], 1.6, Ops::mulc(Lam[5], 0.8))));
    K[52] = Ops::fmac(Lam[9], 1.6, Ops::fmac(Lam[6], 1.6, Ops::mulc(Lam[4], 1.6)));
    K[53] = Ops::fmac(Lam[9], 0.8, Ops::fmac(Lam[8], 0.8, Ops::fmac(Lam[6], 0.8, Ops::mulc(Lam[5], 1.6))));
    K[54] = Ops::fmac(Lam[9], 1.6, Ops::fmac(Lam[8], 1.6, Ops::mulc(Lam[7], 1.6)));
  }
  template <class Ops> __device__ __forceinline__ static void mass_upper_add(const typename Ops::T& vol, typename Ops::T* K) {
    K[0] = Ops::fmac(vol, 0.014285714285714285, K[0]);
    K[1] = Ops::fmac(vol, 0.002380952380952381, K[1]);
    K[2] = Ops::fmac(vol, 0.002380952380952381, K[2]);
    K[3] = Ops::fmac(vol, 0.002380952380952381, K[3]);
    K[4] = Ops::fmac(vol, -0.009523809523809525, K[4]);
    K[5] = Ops::fmac(vol, -0.009523809523809525, K[5]);
    K[6] = Ops::fmac(vol, -0.009523809523809525, K[6]);
    K[7] = Ops::fmac(vol, -0.014285714285714285, K[7]);
    K[8] = Ops::fmac(vol, -0.014285714285714285, K[8]);
    K[9] = Ops::fmac(vol, -0.014285714285714285, K[9]);
    K[10] = Ops::fmac(vol, 0.014285714285714285, K[10]);
    K[11] = Ops::fmac(vol, 0.002380952380952381, K[11]);
    K[12] = Ops::fmac(vol, 0.002380952380952381, K[12]);
    K[13] = Ops::fmac(vol, -0.009523809523809525, K[13]);
    K[14] = Ops::fmac(vol, -0.014285714285714285, K[14]);
    K[15] = Ops::fmac(vol, -0.014285714285714285, K[15]);
    K[16] = Ops::fmac(vol, -0.009523809523809525, K[16]);
    K[17] = Ops::fmac(vol, -0.009523809523809525, K[17]);
    K[18] = Ops::fmac(vol, -0.014285714285714285, K[18]);
    K[19] = Ops::fmac(vol, 0.014285714285714285, K[19]);
    K[20] = Ops::fmac(vol, 0.002380952380952381, K[20]);
    K[21] = Ops::fmac(vol, -0.014285714285714285, K[21]);
    K[22] = Ops::fmac(vol, -0.009523809523809525, K[22]);
    K[23] = Ops::fmac(vol, -0.014285714285714285, K[23]);
    K[24] = Ops::fmac(vol, -0.009523809523809525, K[24]);
    K[25] = Ops::fmac(vol, -0.014285714285714285, K[25]);
    K[26] = Ops::fmac(vol, -0.009523809523809525, K[26]);
    K[27] = Ops::fmac(vol, 0.014285714285714285, K[27]);
    K[28] = Ops::fmac(vol, -0.014285714285714285, K[28]);
    K[29] = Ops::fmac(vol, -0.014285714285714285, K[29]);
    K[30] = Ops::fmac(vol, -0.009523809523809525, K[30]);
    K[31] = Ops::fmac(vol, -0.014285714285714285, K[31]);
    K[32] = Ops::fmac(vol, -0.009523809523809525, K[32]);
    K[33] = Ops::fmac(vol, -0.009523809523809525, K[33]);
    K[34] = Ops::fmac(vol, 0.0761904761904762, K[34]);
    K[35] = Ops::fmac(vol, 0.0380952380952381, K[35]);
    K[36] = Ops::fmac(vol, 0.0380952380952381, K[36]);
    K[37] = Ops::fmac(vol, 0.0380952380952381, K[37]);
    K[38] = Ops::fmac(vol, 0.0380952380952381, K[38]);
    K[39] = Ops::fmac(vol, 0.01904761904761905, K[39]);
    K[40] = Ops::fmac(vol, 0.0761904761904762, K[40]);
    K[41] = Ops::fmac(vol, 0.0380952380952381, K[41]);
    K[42] = Ops::fmac(vol, 0.0380952380952381, K[42]);
    K[43] = Ops::fmac(vol, 0.01904761904761905, K[43]);
    K[44] = Ops::fmac(vol, 0.0380952380952381, K[44]);
    K[45] = Ops::fmac(vol, 0.0761904761904762, K[45]);
    K[46] = Ops::fmac(vol, 0.01904761904761905, K[46]);
    K[47] = Ops::fmac(vol, 0.0380952380952381, K[47]);
    K[48] = Ops::fmac(vol, 0.0380952380952381, K[48]);
    K[49] = Ops::fmac(vol, 0.0761904761904762, K[49]);
    K[50] = Ops::fmac(vol, 0.0380952380952381, K[50]);
    K[51] = Ops::fmac(vol, 0.0380952380952381, K[51]);
    K[52] = Ops::fmac(vol, 0.0761904761904762, K[52]);
    K[53] = Ops::fmac(vol, 0.0380952380952381, K[53]);
    K[54] = Ops::fmac(vol, 0.0761904761904762, K[54]);
  }
  template <class Ops> __device__ __forceinline__ static void mass_upper(const typename Ops::T& vol, typename Ops::T* K) {
    K[0] = Ops::mulc(vol, 0.014285714285714285);
    K[1] = Ops::mulc(vol, 0.002380952380952381);
    K[2] = Ops::mulc(vol, 0.002380952380952381);
    K[3] = Ops::mulc(vol, 0.002380952380952381);
    K[4] = Ops::mulc(vol, -0.009523809523809525);
    K[5] = Ops::mulc(vol, -0.009523809523809525);
    K[6] = Ops::mulc(vol, -0.009523809523809525);
    K[7] = Ops::mulc(vol, -0.014285714285714285);
    K[8] = Ops::mulc(vol, -0.014285714285714285);
    K[9] = Ops::mulc(vol, -0.014285714285714285);
    K[10] = Ops::mulc(vol, 0.014285714285714285);
    K[11] = Ops::mulc(vol, 0.002380952380952381);
    K[12] = Ops::mulc(vol, 0.002380952380952381);
    K[13] = Ops::mulc(vol, -0.009523809523809525);
    K[14] = Ops::mulc(vol, -0.014285714285714285);
    K[15] = Ops::mulc(vol, -0.014285714285714285);
    K[16] = Ops::mulc(vol, -0.009523809523809525);
    K[17] = Ops::mulc(vol, -0.009523809523809525);
    K[18] = Ops::mulc(vol, -0.014285714285714285);
    K[19] = Ops::mulc(vol, 0.014285714285714285);
    K[20] = Ops::mulc(vol, 0.002380952380952381);
    K[21] = Ops::mulc(vol, -0.014285714285714285);
    K[22] = Ops::mulc(vol, -0.009523809523809525);
    K[23] = Ops::mulc(vol, -0.014285714285714285);
    K[24] = Ops::mulc(vol, -0.009523809523809525);
    K[25] = Ops::mulc(vol, -0.014285714285714285);
    K[26] = Ops::mulc(vol, -0.009523809523809525);
    K[27] = Ops::mulc(vol, 0.014285714285714285);
    K[28] = Ops::mulc(vol, -0.014285714285714285);
    K[29] = Ops::mulc(vol, -0.014285714285714285);
    K[30] = Ops::mulc(vol, -0.009523809523809525);
    K[31] = Ops::mulc(vol, -0.014285714285714285);
    K[32] = Ops::mulc(vol, -0.009523809523809525);
    K[33] = Ops::mulc(vol, -0.009523809523809525);
    K[34] = Ops::mulc(vol, 0.0761904761904762);
    K[35] = Ops::mulc(vol, 0.0380952380952381);
    K[36] = Ops::mulc(vol, 0.0380952380952381);
    K[37] = Ops::mulc(vol, 0.0380952380952381);
    K[38] = Ops::mulc(vol, 0.0380952380952381);
    K[39] = Ops::mulc(vol, 0.01904761904761905);
    K[40] = Ops::mulc(vol, 0.0761904761904762);
    K[41] = Ops::mulc(vol, 0.0380952380952381);
    K[42] = Ops::mulc(vol, 0.0380952380952381);
    K[43] = Ops::mulc(vol, 0.01904761904761905);
    K[44] = Ops::mulc(vol, 0.0380952380952381);
    K[45] = Ops::mulc(vol, 0.0761904761904762);
    K[46] = Ops::mulc(vol, 0.01904761904761905);
    K[47] = Ops::mulc(vol, 0.0380952380952381);
    K[48] = Ops::mulc(vol, 0.0380952380952381);
    K[49] = Ops::mulc(vol, 0.0761904761904762);
    K[50] = Ops::mulc(vol, 0.0380952380952381);
    K[51] = Ops::mulc(vol, 0.0380952380952381);
    K[52] = Ops::mulc(vol, 0.0761904761904762);
    K[53] = Ops::mulc(vol, 0.0380952380952381);
    K[54] = Ops::mulc(vol, 0.0761904761904762);
  }
  template <class Ops, bool STIFF, bool MASS> __device__ __forceinline__ static void action_upper(const typename Ops::T* Lam, const typename Ops::T& vol, const typename Ops::T* x, typename Ops::T* y) {
    typename Ops::T k;
    { if constexpr (STIFF) { k = Ops::mulc(Lam[0], 0.6); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, 0.014285714285714285, k); } y[0] = Ops::fma3(k, x[0], y[0]); }
    { if constexpr (STIFF) { k = Ops::mulc(Lam[1], -0.2); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, 0.002380952380952381, k); } y[0] = Ops::fma3(k, x[1], y[0]); y[1] = Ops::fma3(k, x[0], y[1]); }
    { if constexpr (STIFF) { k = Ops::mulc(Lam[2], -0.2); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, 0.002380952380952381, k); } y[0] = Ops::fma3(k, x[2], y[0]); y[2] = Ops::fma3(k, x[0], y[2]); }
    { if constexpr (STIFF) { k = Ops::mulc(Lam[3], -0.2); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, 0.002380952380952381, k); } y[0] = Ops::fma3(k, x[3], y[0]); y[3] = Ops::fma3(k, x[0], y[3]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[1], 0.6, Ops::mulc(Lam[0], -0.2)); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, -0.009523809523809525, k); } y[0] = Ops::fma3(k, x[4], y[0]); y[4] = Ops::fma3(k, x[0], y[4]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[2], 0.6, Ops::mulc(Lam[0], -0.2)); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, -0.009523809523809525, k); } y[0] = Ops::fma3(k, x[5], y[0]); y[5] = Ops::fma3(k, x[0], y[5]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[3], 0.6, Ops::mulc(Lam[0], -0.2)); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, -0.009523809523809525, k); } y[0] = Ops::fma3(k, x[6], y[0]); y[6] = Ops::fma3(k, x[0], y[6]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[2], -0.2, Ops::mulc(Lam[1], -0.2)); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, -0.014285714285714285, k); } y[0] = Ops::fma3(k, x[7], y[0]); y[7] = Ops::fma3(k, x[0], y[7]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[3], -0.2, Ops::mulc(Lam[1], -0.2)); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, -0.014285714285714285, k); } y[0] = Ops::fma3(k, x[8], y[0]); y[8] = Ops::fma3(k, x[0], y[8]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[3], -0.2, Ops::mulc(Lam[2], -0.2)); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, -0.014285714285714285, k); } y[0] = Ops::fma3(k, x[9], y[0]); y[9] = Ops::fma3(k, x[0], y[9]); }
    { if constexpr (STIFF) { k = Ops::mulc(Lam[4], 0.6); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, 0.014285714285714285, k); } y[1] = Ops::fma3(k, x[1], y[1]); }
    { if constexpr (STIFF) { k = Ops::mulc(Lam[5], -0.2); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, 0.002380952380952381, k); } y[1] = Ops::fma3(k, x[2], y[1]); y[2] = Ops::fma3(k, x[1], y[2]); }
    { if constexpr (STIFF) { k = Ops::mulc(Lam[6], -0.2); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, 0.002380952380952381, k); } y[1] = Ops::fma3(k, x[3], y[1]); y[3] = Ops::fma3(k, x[1], y[3]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[4], -0.2, Ops::mulc(Lam[1], 0.6)); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, -0.009523809523809525, k); } y[1] = Ops::fma3(k, x[4], y[1]); y[4] = Ops::fma3(k, x[1], y[4]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[5], -0.2, Ops::mulc(Lam[1], -0.2)); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, -0.014285714285714285, k); } y[1] = Ops::fma3(k, x[5], y[1]); y[5] = Ops::fma3(k, x[1], y[5]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[6], -0.2, Ops::mulc(Lam[1], -0.2)); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, -0.014285714285714285, k); } y[1] = Ops::fma3(k, x[6], y[1]); y[6] = Ops::fma3(k, x[1], y[6]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[5], 0.6, Ops::mulc(Lam[4], -0.2)); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, -0.009523809523809525, k); } y[1] = Ops::fma3(k, x[7], y[1]); y[7] = Ops::fma3(k, x[1], y[7]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[6], 0.6, Ops::mulc(Lam[4], -0.2)); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, -0.009523809523809525, k); } y[1] = Ops::fma3(k, x[8], y[1]); y[8] = Ops::fma3(k, x[1], y[8]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[6], -0.2, Ops::mulc(Lam[5], -0.2)); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, -0.014285714285714285, k); } y[1] = Ops::fma3(k, x[9], y[1]); y[9] = Ops::fma3(k, x[1], y[9]); }
    { if constexpr (STIFF) { k = Ops::mulc(Lam[7], 0.6); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, 0.014285714285714285, k); } y[2] = Ops::fma3(k, x[2], y[2]); }
    { if constexpr (STIFF) { k = Ops::mulc(Lam[8], -0.2); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, 0.002380952380952381, k); } y[2] = Ops::fma3(k, x[3], y[2]); y[3] = Ops::fma3(k, x[2], y[3]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[5], -0.2, Ops::mulc(Lam[2], -0.2)); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, -0.014285714285714285, k); } y[2] = Ops::fma3(k, x[4], y[2]); y[4] = Ops::fma3(k, x[2], y[4]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[7], -0.2, Ops::mulc(Lam[2], 0.6)); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, -0.009523809523809525, k); } y[2] = Ops::fma3(k, x[5], y[2]); y[5] = Ops::fma3(k, x[2], y[5]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[8], -0.2, Ops::mulc(Lam[2], -0.2)); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, -0.014285714285714285, k); } y[2] = Ops::fma3(k, x[6], y[2]); y[6] = Ops::fma3(k, x[2], y[6]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[7], -0.2, Ops::mulc(Lam[5], 0.6)); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, -0.009523809523809525, k); } y[2] = Ops::fma3(k, x[7], y[2]); y[7] = Ops::fma3(k, x[2], y[7]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[8], -0.2, Ops::mulc(Lam[5], -0.2)); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, -0.014285714285714285, k); } y[2] = Ops::fma3(k, x[8], y[2]); y[8] = Ops::fma3(k, x[2], y[8]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[8], 0.6, Ops::mulc(Lam[7], -0.2)); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, -0.009523809523809525, k); } y[2] = Ops::fma3(k, x[9], y[2]); y[9] = Ops::fma3(k, x[2], y[9]); }
    { if constexpr (STIFF) { k = Ops::mulc(Lam[9], 0.6); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, 0.014285714285714285, k); } y[3] = Ops::fma3(k, x[3], y[3]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[6], -0.2, Ops::mulc(Lam[3], -0.2)); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, -0.014285714285714285, k); } y[3] = Ops::fma3(k, x[4], y[3]); y[4] = Ops::fma3(k, x[3], y[4]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[8], -0.2, Ops::mulc(Lam[3], -0.2)); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, -0.014285714285714285, k); } y[3] = Ops::fma3(k, x[5], y[3]); y[5] = Ops::fma3(k, x[3], y[5]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[9], -0.2, Ops::mulc(Lam[3], 0.6)); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, -0.009523809523809525, k); } y[3] = Ops::fma3(k, x[6], y[3]); y[6] = Ops::fma3(k, x[3], y[6]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[8], -0.2, Ops::mulc(Lam[6], -0.2)); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, -0.014285714285714285, k); } y[3] = Ops::fma3(k, x[7], y[3]); y[7] = Ops::fma3(k, x[3], y[7]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[9], -0.2, Ops::mulc(Lam[6], 0.6)); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, -0.009523809523809525, k); } y[3] = Ops::fma3(k, x[8], y[3]); y[8] = Ops::fma3(k, x[3], y[8]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[9], -0.2, Ops::mulc(Lam[8], 0.6)); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, -0.009523809523809525, k); } y[3] = Ops::fma3(k, x[9], y[3]); y[9] = Ops::fma3(k, x[3], y[9]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[4], 1.6, Ops::fmac(Lam[1], 1.6, Ops::mulc(Lam[0], 1.6))); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, 0.0761904761904762, k); } y[4] = Ops::fma3(k, x[4], y[4]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[5], 1.6, Ops::fmac(Lam[2], 0.8, Ops::fmac(Lam[1], 0.8, Ops::mulc(Lam[0], 0.8)))); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, 0.0380952380952381, k); } y[4] = Ops::fma3(k, x[5], y[4]); y[5] = Ops::fma3(k, x[4], y[5]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[6], 1.6, Ops::fmac(Lam[3], 0.8, Ops::fmac(Lam[1], 0.8, Ops::mulc(Lam[0], 0.8)))); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, 0.0380952380952381, k); } y[4] = Ops::fma3(k, x[6], y[4]); y[6] = Ops::fma3(k, x[4], y[6]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[5], 0.8, Ops::fmac(Lam[4], 0.8, Ops::fmac(Lam[2], 1.6, Ops::mulc(Lam[1], 0.8)))); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, 0.0380952380952381, k); } y[4] = Ops::fma3(k, x[7], y[4]); y[7] = Ops::fma3(k, x[4], y[7]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[6], 0.8, Ops::fmac(Lam[4], 0.8, Ops::fmac(Lam[3], 1.6, Ops::mulc(Lam[1], 0.8)))); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, 0.0380952380952381, k); } y[4] = Ops::fma3(k, x[8], y[4]); y[8] = Ops::fma3(k, x[4], y[8]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[6], 0.8, Ops::fmac(Lam[5], 0.8, Ops::fmac(Lam[3], 0.8, Ops::mulc(Lam[2], 0.8)))); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, 0.01904761904761905, k); } y[4] = Ops::fma3(k, x[9], y[4]); y[9] = Ops::fma3(k, x[4], y[9]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[7], 1.6, Ops::fmac(Lam[2], 1.6, Ops::mulc(Lam[0], 1.6))); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, 0.0761904761904762, k); } y[5] = Ops::fma3(k, x[5], y[5]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[8], 1.6, Ops::fmac(Lam[3], 0.8, Ops::fmac(Lam[2], 0.8, Ops::mulc(Lam[0], 0.8)))); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, 0.0380952380952381, k); } y[5] = Ops::fma3(k, x[6], y[5]); y[6] = Ops::fma3(k, x[5], y[6]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[7], 0.8, Ops::fmac(Lam[5], 0.8, Ops::fmac(Lam[2], 0.8, Ops::mulc(Lam[1], 1.6)))); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, 0.0380952380952381, k); } y[5] = Ops::fma3(k, x[7], y[5]); y[7] = Ops::fma3(k, x[5], y[7]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[8], 0.8, Ops::fmac(Lam[5], 0.8, Ops::fmac(Lam[3], 0.8, Ops::mulc(Lam[1], 0.8)))); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, 0.01904761904761905, k); } y[5] = Ops::fma3(k, x[8], y[5]); y[8] = Ops::fma3(k, x[5], y[8]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[8], 0.8, Ops::fmac(Lam[7], 0.8, Ops::fmac(Lam[3], 1.6, Ops::mulc(Lam[2], 0.8)))); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, 0.0380952380952381, k); } y[5] = Ops::fma3(k, x[9], y[5]); y[9] = Ops::fma3(k, x[5], y[9]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[9], 1.6, Ops::fmac(Lam[3], 1.6, Ops::mulc(Lam[0], 1.6))); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, 0.0761904761904762, k); } y[6] = Ops::fma3(k, x[6], y[6]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[8], 0.8, Ops::fmac(Lam[6], 0.8, Ops::fmac(Lam[2], 0.8, Ops::mulc(Lam[1], 0.8)))); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, 0.01904761904761905, k); } y[6] = Ops::fma3(k, x[7], y[6]); y[7] = Ops::fma3(k, x[6], y[7]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[9], 0.8, Ops::fmac(Lam[6], 0.8, Ops::fmac(Lam[3], 0.8, Ops::mulc(Lam[1], 1.6)))); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, 0.0380952380952381, k); } y[6] = Ops::fma3(k, x[8], y[6]); y[8] = Ops::fma3(k, x[6], y[8]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[9], 0.8, Ops::fmac(Lam[8], 0.8, Ops::fmac(Lam[3], 0.8, Ops::mulc(Lam[2], 1.6)))); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, 0.0380952380952381, k); } y[6] = Ops::fma3(k, x[9], y[6]); y[9] = Ops::fma3(k, x[6], y[9]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[7], 1.6, Ops::fmac(Lam[5], 1.6, Ops::mulc(Lam[4], 1.6))); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, 0.0761904761904762, k); } y[7] = Ops::fma3(k, x[7], y[7]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[8], 1.6, Ops::fmac(Lam[6], 0.8, Ops::fmac(Lam[5], 0.8, Ops::mulc(Lam[4], 0.8)))); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, 0.0380952380952381, k); } y[7] = Ops::fma3(k, x[8], y[7]); y[8] = Ops::fma3(k, x[7], y[8]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[8], 0.8, Ops::fmac(Lam[7], 0.8, Ops::fmac(Lam[6], 1.6, Ops::mulc(Lam[5], 0.8)))); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, 0.0380952380952381, k); } y[7] = Ops::fma3(k, x[9], y[7]); y[9] = Ops::fma3(k, x[7], y[9]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[9], 1.6, Ops::fmac(Lam[6], 1.6, Ops::mulc(Lam[4], 1.6))); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, 0.0761904761904762, k); } y[8] = Ops::fma3(k, x[8], y[8]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[9], 0.8, Ops::fmac(Lam[8], 0.8, Ops::fmac(Lam[6], 0.8, Ops::mulc(Lam[5], 1.6)))); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, 0.0380952380952381, k); } y[8] = Ops::fma3(k, x[9], y[8]); y[9] = Ops::fma3(k, x[8], y[9]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[9], 1.6, Ops::fmac(Lam[8], 1.6, Ops::mulc(Lam[7], 1.6))); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, 0.0761904761904762, k); } y[9] = Ops::fma3(k, x[9], y[9]); }
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
  template <class Ops> __device__ __forceinline__ static void stiffness_upper(const typename Ops::T* Lam, typename Ops::T* K) {
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
    K[10] = Ops::fmac(Lam[2], 0.08035714285714286, Ops::mulc(Lam[1], 0.08035714285714286));
    K[11] = Ops::fmac(Lam[2], 0.08035714285714286, Ops::mulc(Lam[1], 0.08035714285714286));
    K[12] = Ops::fmac(Lam[3], 0.08035714285714286, Ops::mulc(Lam[1], 0.08035714285714286));
    K[13] = Ops::fmac(Lam[3], 0.08035714285714286, Ops::mulc(Lam[1], 0.08035714285714286));
    K[14] = Ops::fmac(Lam[3], 0.08035714285714286, Ops::mulc(Lam[2], 0.08035714285714286));
    K[15] = Ops::fmac(Lam[3], 0.08035714285714286, Ops::mulc(Lam[2], 0.08035714285714286));
    K[16] = Ops::fmac(Lam[2], -0.09642857142857143, Ops::fmac(Lam[1], -0.09642857142857143, Ops::mulc(Lam[0], 0.19285714285714287)));
    K[17] = Ops::fmac(Lam[3], -0.09642857142857143, Ops::fmac(Lam[1], -0.09642857142857143, Ops::mulc(Lam[0], 0.19285714285714287)));
    K[18] = Ops::fmac(Lam[3], -0.09642857142857143, Ops::fmac(Lam[2], -0.09642857142857143, Ops::mulc(Lam[0], 0.19285714285714287)));
    K[19] = Ops::fmac(Lam[3], 0.19285714285714287, Ops::fmac(Lam[2], 0.19285714285714287, Ops::mulc(Lam[1], 0.19285714285714287)));
    K[20] = Ops::mulc(Lam[4], 0.35714285714285715);
    K[21] = Ops::mulc(Lam[5], 0.06785714285714285);
    K[22] = Ops::mulc(Lam[6], 0.06785714285714285);
    K[23] = Ops::fmac(Lam[4], 0.08035714285714286, Ops::mulc(Lam[1], -0.20892857142857144));
    K[24] = Ops::fmac(Lam[4], -0.20892857142857144, Ops::mulc(Lam[1], 0.36964285714285716));
    K[25] = Ops::fmac(Lam[5], 0.08035714285714286, Ops::mulc(Lam[1], 0.08035714285714286));
    K[26] = Ops::fmac(Lam[5], 0.08035714285714286, Ops::mulc(Lam[1], 0.08035714285714286));
    K[27] = Ops::fmac(Lam[6], 0.08035714285714286, Ops::mulc(Lam[1], 0.08035714285714286));
    K[28] = Ops::fmac(Lam[6], 0.08035714285714286, Ops::mulc(Lam[1], 0.08035714285714286));
    K[29] = Ops::fmac(Lam[5], 0.36964285714285716, Ops::mulc(Lam[4], -0.20892857142857144));
    K[30] = Ops::fmac(Lam[5], -0.20892857142857144, Ops::mulc(Lam[4], 0.08035714285714286));
    K[31] = Ops::fmac(Lam[6], 0.36964285714285716, Ops::mulc(Lam[4], -0.20892857142857144));
    K[32] = Ops::fmac(Lam[6], -0.20892857142857144, Ops::mulc(Lam[4], 0.08035714285714286));
    K[33] = Ops::fmac(Lam[6], 0.08035714285714286, Ops::mulc(Lam[5], 0.08035714285714286));
    K[34] = Ops::fmac(Lam[6], 0.08035714285714286, Ops::mulc(Lam[5], 0.08035714285714286));
    K[35] = Ops::fmac(Lam[5], -0.09642857142857143, Ops::fmac(Lam[4], 0.19285714285714287, Ops::mulc(Lam[1], -0.09642857142857143)));
    K[36] = Ops::fmac(Lam[6], -0.09642857142857143, Ops::fmac(Lam[4], 0.19285714285714287, Ops::mulc(Lam[1], -0.09642857142857143)));
    K[37] = Ops::fmac(Lam[6], 0.19285714285714287, Ops::fmac(Lam[5], 0.19285714285714287, Ops::mulc(Lam[1], 0.19285714285714287)));
    K[38] = Ops::fmac(Lam[6], -0.09642857142857143, Ops::fmac(Lam[5], -0.09642857142857143, Ops::mulc(Lam[4], 0.19285714285714287)));
    K[39] = Ops::mulc(Lam[7], 0.35714285714285715);
    K[40] = Ops::mulc(Lam[8], 0.06785714285714285);
    K[41] = Ops::fmac(Lam[5], 0.08035714285714286, Ops::mulc(Lam[2], 0.08035714285714286));
    K[42] = Ops::fmac(Lam[5], 0.08035714285714286, Ops::mulc(Lam[2], 0.08035714285714286));
    K[43] = Ops::fmac(Lam[7], 0.08035714285714286, Ops::mulc(Lam[2], -0.20892857142857144));
    K[44] = Ops::fmac(Lam[7], -0.20892857142857144, Ops::mulc(Lam[2], 0.36964285714285716));
    K[45] = Ops::fmac(Lam[8], 0.08035714285714286, Ops::mulc(Lam[2], 0.08035714285714286));
    K[46] = Ops::fmac(Lam[8], 0.08035714285714286, Ops::mulc(Lam[2], 0.08035714285714286));
    K[47] = Ops::fmac(Lam[7], 0.08035714285714286, Ops::mulc(Lam[5], -0.20892857142857144));
    K[48] = Ops::fmac(Lam[7], -0.20892857142857144, Ops::mulc(Lam[5], 0.36964285714285716));
    K[49] = Ops::fmac(Lam[8], 0.08035714285714286, Ops::mulc(Lam[5], 0.08035714285714286));
    K[50] = Ops::fmac(Lam[8], 0.08035714285714286, Ops::mulc(Lam[5], 0.08035714285714286));
    K[51] = Ops::fmac(Lam[8], 0.36964285714285716, Ops::mulc(Lam[7], -0.20892857142857144));
    K[52] = Ops::fmac(Lam[8], -0.20892857142857144, Ops::mulc(Lam[7], 0.08035714285714286));
    K[53] = Ops::fmac(Lam[7], 0.19285714285714287, Ops::fmac(Lam[5], -0.09642857142857143, Ops::mulc(Lam[2], -0.09642857142857143)));
    K[54] = Ops::fmac(Lam[8], 0.19285714285714287, Ops::fmac(Lam[5], 0.19285714285714287, Ops::mulc(Lam[2], 0.19285714285714287)));
    K[55] = Ops::fmac(Lam[8], -0.09642857142857143, Ops::fmac(Lam[7], 0.19285714285714287, Ops::mulc(Lam[2], -0.09642857142857143)));
    K[56] = Ops::fmac(Lam[8], -0.09642857142857143, Ops::fmac(Lam[7], 0.19285714285714287, Ops::mulc(Lam[5], -0.09642857142857143)));
    K[57] = Ops::mulc(Lam[9], 0.35714285714285715);
    K[58] = Ops::fmac(Lam[6], 0.08035714285714286, Ops::mulc(Lam[3], 0.08035714285714286));
    K[59] = Ops::fmac(Lam[6], 0.08035714285714286, Ops::mulc(Lam[3], 0.08035714285714286));
    K[60] = Ops::fmac(Lam[8], 0.08035714285714286, Ops::mulc(Lam[3], 0.08035714285714286));
    K[61] = Ops::fmac(Lam[8], 0.08035714285714286, Ops::mulc(Lam[3], 0.08035714285714286));
    K[62] = Ops::fmac(Lam[9], 0.08035714285714286, Ops::mulc(Lam[3], -0.20892857142857144));
    K[63] = Ops::fmac(Lam[9], -0.20892857142857144, Ops::mulc(Lam[3], 0.36964285714285716));
    K[64] = Ops::fmac(Lam[8], 0.08035714285714286, Ops::mulc(Lam[6], 0.08035714285714286));
    K[65] = Ops::fmac(Lam[8], 0.08035714285714286, Ops::mulc(Lam[6], 0.08035714285714286));
    K[66] = Ops::fmac(Lam[9], 0.08035714285714286, Ops::mulc(Lam[6], -0.20892857142857144));
    K[67] = Ops::fmac(Lam[9], -0.20892857142857144, Ops::mulc(Lam[6], 0.36964285714285716));
    K[68] = Ops::fmac(Lam[9], 0.08035714285714286, Ops::mulc(Lam[8], -0.20892857142857144));
    K[69] = Ops::fmac(Lam[9], -0.20892857142857144, Ops::mulc(Lam[8], 0.36964285714285716));
    K[70] = Ops::fmac(Lam[8], 0.19285714285714287, Ops::fmac(Lam[6], 0.19285714285714287, Ops::mulc(Lam[3], 0.19285714285714287)));
    K[71] = Ops::fmac(Lam[9], 0.19285714285714287, Ops::fmac(Lam[6], -0.09642857142857143, Ops::mulc(Lam[3], -0.09642857142857143)));
    K[72] = Ops::fmac(Lam[9], 0.19285714285714287, Ops::fmac(Lam[8], -0.09642857142857143, Ops::mulc(Lam[3], -0.09642857142857143)));
    K[73] = Ops::fmac(Lam[9], 0.19285714285714287, Ops::fmac(Lam[8], -0.09642857142857143, Ops::mulc(Lam[6], -0.09642857142857143)));
    K[74] = Ops::fmac(Lam[4], 1.1571428571428573, Ops::fmac(Lam[1], 1.1571428571428573, Ops::mulc(Lam[0], 1.4464285714285714)));
    K[75] = Ops::fmac(Lam[4], -0.43392857142857144, Ops::fmac(Lam[1], 0.2892857142857143, Ops::mulc(Lam[0], -0.43392857142857144)));
    K[76] = Ops::fmac(Lam[5], 1.1571428571428573, Ops::fmac(Lam[2], 0.5785714285714286, Ops::fmac(Lam[1], 0.5785714285714286, Ops::mulc(Lam[0], 0.7232142857142857))));
    K[77] = Ops::fmac(Lam[5], -0.43392857142857144, Ops::fmac(Lam[2], -0.2892857142857143, Ops::fmac(Lam[1], -0.14464285714285716, Ops::mulc(Lam[0], -0.14464285714285716))));
    K[78] = Ops::fmac(Lam[6], 1.1571428571428573, Ops::fmac(Lam[3], 0.5785714285714286, Ops::fmac(Lam[1], 0.5785714285714286, Ops::mulc(Lam[0], 0.7232142857142857))));
    K[79] = Ops::fmac(Lam[6], -0.43392857142857144, Ops::fmac(Lam[3], -0.2892857142857143, Ops::fmac(Lam[1], -0.14464285714285716, Ops::mulc(Lam[0], -0.14464285714285716))));
    K[80] = Ops::fmac(Lam[5], -0.14464285714285716, Ops::fmac(Lam[4], -0.14464285714285716, Ops::fmac(Lam[2], -0.43392857142857144, Ops::mulc(Lam[1], -0.2892857142857143))));
    K[81] = Ops::fmac(Lam[5], -0.14464285714285716, Ops::fmac(Lam[4], -0.14464285714285716, Ops::fmac(Lam[2], -0.2892857142857143, Ops::mulc(Lam[1], -0.14464285714285716))));
    K[82] = Ops::fmac(Lam[6], -0.14464285714285716, Ops::fmac(Lam[4], -0.14464285714285716, Ops::fmac(Lam[3], -0.43392857142857144, Ops::mulc(Lam[1], -0.2892857142857143))));
    K[83] = Ops::fmac(Lam[6], -0.14464285714285716, Ops::fmac(Lam[4], -0.14464285714285716, Ops::fmac(Lam[3], -0.2892857142857143, Ops::mulc(Lam[1], -0.14464285714285716))));
    K[84] = Ops::fmac(Lam[6], -0.14464285714285716, Ops::fmac(Lam[5], -0.14464285714285716, Ops::fmac(Lam[3], -0.14464285714285716, Ops::mulc(Lam[2], -0.14464285714285716))));
    K[85] = Ops::fmac(Lam[6], -0.14464285714285716, Ops::fmac(Lam[5], -0.14464285714285716, Ops::fmac(Lam[3], -0.14464285714285716, Ops::mulc(Lam[2], -0.14464285714285716))));
    K[86] = Ops::fmac(Lam[5], 0.5785714285714286, Ops::fmac(Lam[4], 0.5785714285714286, Ops::fmac(Lam[2], 1.4464285714285714, Ops::fmac(Lam[1], 0.5785714285714286, Ops::mulc(Lam[0], -0.2892857142857143)))));
    K[87] = Ops::fmac(Lam[6], 0.5785714285714286, Ops::fmac(Lam[4], 0.5785714285714286, Ops::fmac(Lam[3], 1.4464285714285714, Ops::fmac(Lam[1], 0.5785714285714286, Ops::mulc(Lam[0], -0.2892857142857143)))));
    K[88] = Ops::fmac(Lam[6], 0.5785714285714286, Ops::fmac(Lam[5], 0.5785714285714286, Ops::fmac(Lam[3], 0.7232142857142857, Ops::fmac(Lam[2], 0.7232142857142857, Ops::fmac(Lam[1], -0.14464285714285716, Ops::mulc(Lam[0], -0.14464285714285716))))));
    K[89] = Ops::fmac(Lam[6], -0.14464285714285716, Ops::fmac(Lam[5], -0.14464285714285716, Ops::fmac(Lam[4], -0.14464285714285716, Ops::fmac(Lam[3], -0.2892857142857143, Ops::fmac(Lam[2], -0.2892857142857143, Ops::mulc(Lam[1], -0.14464285714285716))))));
    K[90] = Ops::fmac(Lam[4], 1.4464285714285714, Ops::fmac(Lam[1], 1.1571428571428573, Ops::mulc(Lam[0], 1.1571428571428573)));
    K[91] = Ops::fmac(Lam[5], -0.43392857142857144, Ops::fmac(Lam[2], -0.14464285714285716, Ops::fmac(Lam[1], -0.2892857142857143, Ops::mulc(Lam[0], -0.14464285714285716))));
    K[92] = Ops::fmac(Lam[5], -0.2892857142857143, Ops::fmac(Lam[2], -0.14464285714285716, Ops::fmac(Lam[1], -0.14464285714285716, Ops::mulc(Lam[0], -0.14464285714285716))));
    K[93] = Ops::fmac(Lam[6], -0.43392857142857144, Ops::fmac(Lam[3], -0.14464285714285716, Ops::fmac(Lam[1], -0.2892857142857143, Ops::mulc(Lam[0], -0.14464285714285716))));
    K[94] = Ops::fmac(Lam[6], -0.2892857142857143, Ops::fmac(Lam[3], -0.14464285714285716, Ops::fmac(Lam[1], -0.14464285714285716, Ops::mulc(Lam[0], -0.14464285714285716))));
    K[95] = Ops::fmac(Lam[5], 0.5785714285714286, Ops::fmac(Lam[4], 0.7232142857142857, Ops::fmac(Lam[2], 1.1571428571428573, Ops::mulc(Lam[1], 0.5785714285714286))));
    K[96] = Ops::fmac(Lam[5], -0.2892857142857143, Ops::fmac(Lam[4], -0.14464285714285716, Ops::fmac(Lam[2], -0.43392857142857144, Ops::mulc(Lam[1], -0.14464285714285716))));
    K[97] = Ops::fmac(Lam[6], 0.5785714285714286, Ops::fmac(Lam[4], 0.7232142857142857, Ops::fmac(Lam[3], 1.1571428571428573, Ops::mulc(Lam[1], 0.5785714285714286))));
    K[98] = Ops::fmac(Lam[6], -0.2892857142857143, Ops::fmac(Lam[4], -0.14464285714285716, Ops::fmac(Lam[3], -0.43392857142857144, Ops::mulc(Lam[1], -0.14464285714285716))));
    K[99] = Ops::fmac(Lam[6], -0.14464285714285716, Ops::fmac(Lam[5], -0.14464285714285716, Ops::fmac(Lam[3], -0.14464285714285716, Ops::mulc(Lam[2], -0.14464285714285716))));
    K[100] = Ops::fmac(Lam[6], -0.14464285714285716, Ops::fmac(Lam[5], -0.14464285714285716, Ops::fmac(Lam[3], -0.14464285714285716, Ops::mulc(Lam[2], -0.14464285714285716))));
    K[101] = Ops::fmac(Lam[5], 1.4464285714285714, Ops::fmac(Lam[4], -0.2892857142857143, Ops::fmac(Lam[2], 0.5785714285714286, Ops::fmac(Lam[1], 0.5785714285714286, Ops::mulc(Lam[0], 0.5785714285714286)))));
    K[102] = Ops::fmac(Lam[6], 1.4464285714285714, Ops::fmac(Lam[4], -0.2892857142857143, Ops::fmac(Lam[3], 0.5785714285714286, Ops::fmac(Lam[1], 0.5785714285714286, Ops::mulc(Lam[0], 0.5785714285714286)))));
    K[103] = Ops::fmac(Lam[6], -0.2892857142857143, Ops::fmac(Lam[5], -0.2892857142857143, Ops::fmac(Lam[3], -0.14464285714285716, Ops::fmac(Lam[2], -0.14464285714285716, Ops::fmac(Lam[1], -0.14464285714285716, Ops::mulc(Lam[0], -0.14464285714285716))))));
    K[104] = Ops::fmac(Lam[6], 0.7232142857142857, Ops::fmac(Lam[5], 0.7232142857142857, Ops::fmac(Lam[4], -0.14464285714285716, Ops::fmac(Lam[3], 0.5785714285714286, Ops::fmac(Lam[2], 0.5785714285714286, Ops::mulc(Lam[1], -0.14464285714285716))))));
    K[105] = Ops::fmac(Lam[7], 1.1571428571428573, Ops::fmac(Lam[2], 1.1571428571428573, Ops::mulc(Lam[0], 1.4464285714285714)));
    K[106] = Ops::fmac(Lam[7], -0.43392857142857144, Ops::fmac(Lam[2], 0.2892857142857143, Ops::mulc(Lam[0], -0.43392857142857144)));
    K[107] = Ops::fmac(Lam[8], 1.1571428571428573, Ops::fmac(Lam[3], 0.5785714285714286, Ops::fmac(Lam[2], 0.5785714285714286, Ops::mulc(Lam[0], 0.7232142857142857))));
    K[108] = Ops::fmac(Lam[8], -0.43392857142857144, Ops::fmac(Lam[3], -0.2892857142857143, Ops::fmac(Lam[2], -0.14464285714285716, Ops::mulc(Lam[0], -0.14464285714285716))));
    K[109] = Ops::fmac(Lam[7], -0.14464285714285716, Ops::fmac(Lam[5], -0.14464285714285716, Ops::fmac(Lam[2], -0.14464285714285716, Ops::mulc(Lam[1], -0.2892857142857143))));
    K[110] = Ops::fmac(Lam[7], -0.14464285714285716, Ops::fmac(Lam[5], -0.14464285714285716, Ops::fmac(Lam[2], -0.2892857142857143, Ops::mulc(Lam[1], -0.43392857142857144))));
    K[111] = Ops::fmac(Lam[8], -0.14464285714285716, Ops::fmac(Lam[5], -0.14464285714285716, Ops::fmac(Lam[3], -0.14464285714285716, Ops::mulc(Lam[1], -0.14464285714285716))));
    K[112] = Ops::fmac(Lam[8], -0.14464285714285716, Ops::fmac(Lam[5], -0.14464285714285716, Ops::fmac(Lam[3], -0.14464285714285716, Ops::mulc(Lam[1], -0.14464285714285716))));
    K[113] = Ops::fmac(Lam[8], -0.14464285714285716, Ops::fmac(Lam[7], -0.14464285714285716, Ops::fmac(Lam[3], -0.43392857142857144, Ops::mulc(Lam[2], -0.2892857142857143))));
    K[114] = Ops::fmac(Lam[8], -0.14464285714285716, Ops::fmac(Lam[7], -0.14464285714285716, Ops::fmac(Lam[3], -0.2892857142857143, Ops::mulc(Lam[2], -0.14464285714285716))));
    K[115] = Ops::fmac(Lam[7], 0.5785714285714286, Ops::fmac(Lam[5], 0.5785714285714286, Ops::fmac(Lam[2], 0.5785714285714286, Ops::fmac(Lam[1], 1.4464285714285714, Ops::mulc(Lam[0], -0.2892857142857143)))));
    K[116] = Ops::fmac(Lam[8], 0.5785714285714286, Ops::fmac(Lam[5], 0.5785714285714286, Ops::fmac(Lam[3], 0.7232142857142857, Ops::fmac(Lam[2], -0.14464285714285716, Ops::fmac(Lam[1], 0.7232142857142857, Ops::mulc(Lam[0], -0.14464285714285716))))));
    K[117] = Ops::fmac(Lam[8], 0.5785714285714286, Ops::fmac(Lam[7], 0.5785714285714286, Ops::fmac(Lam[3], 1.4464285714285714, Ops::fmac(Lam[2], 0.5785714285714286, Ops::mulc(Lam[0], -0.2892857142857143)))));
    K[118] = Ops::fmac(Lam[8], -0.14464285714285716, Ops::fmac(Lam[7], -0.14464285714285716, Ops::fmac(Lam[5], -0.14464285714285716, Ops::fmac(Lam[3], -0.2892857142857143, Ops::fmac(Lam[2], -0.14464285714285716, Ops::mulc(Lam[1], -0.2892857142857143))))));
    K[119] = Ops::fmac(Lam[7], 1.4464285714285714, Ops::fmac(Lam[2], 1.1571428571428573, Ops::mulc(Lam[0], 1.1571428571428573)));
    K[120] = Ops::fmac(Lam[8], -0.43392857142857144, Ops::fmac(Lam[3], -0.14464285714285716, Ops::fmac(Lam[2], -0.2892857142857143, Ops::mulc(Lam[0], -0.14464285714285716))));
    K[121] = Ops::fmac(Lam[8], -0.2892857142857143, Ops::fmac(Lam[3], -0.14464285714285716, Ops::fmac(Lam[2], -0.14464285714285716, Ops::mulc(Lam[0], -0.14464285714285716))));
    K[122] = Ops::fmac(Lam[7], -0.14464285714285716, Ops::fmac(Lam[5], -0.2892857142857143, Ops::fmac(Lam[2], -0.14464285714285716, Ops::mulc(Lam[1], -0.43392857142857144))));
    K[123] = Ops::fmac(Lam[7], 0.7232142857142857, Ops::fmac(Lam[5], 0.5785714285714286, Ops::fmac(Lam[2], 0.5785714285714286, Ops::mulc(Lam[1], 1.1571428571428573))));
    K[124] = Ops::fmac(Lam[8], -0.14464285714285716, Ops::fmac(Lam[5], -0.14464285714285716, Ops::fmac(Lam[3], -0.14464285714285716, Ops::mulc(Lam[1], -0.14464285714285716))));
    K[125] = Ops::fmac(Lam[8], -0.14464285714285716, Ops::fmac(Lam[5], -0.14464285714285716, Ops::fmac(Lam[3], -0.14464285714285716, Ops::mulc(Lam[1], -0.14464285714285716))));
    K[126] = Ops::fmac(Lam[8], 0.5785714285714286, Ops::fmac(Lam[7], 0.7232142857142857, Ops::fmac(Lam[3], 1.1571428571428573, Ops::mulc(Lam[2], 0.5785714285714286))));
    K[127] = Ops::fmac(Lam[8], -0.2892857142857143, Ops::fmac(Lam[7], -0.14464285714285716, Ops::fmac(Lam[3], -0.43392857142857144, Ops::mulc(Lam[2], -0.14464285714285716))));
    K[128] = Ops::fmac(Lam[7], -0.2892857142857143, Ops::fmac(Lam[5], 1.4464285714285714, Ops::fmac(Lam[2], 0.5785714285714286, Ops::fmac(Lam[1], 0.5785714285714286, Ops::mulc(Lam[0], 0.5785714285714286)))));
    K[129] = Ops::fmac(Lam[8], -0.2892857142857143, Ops::fmac(Lam[5], -0.2892857142857143, Ops::fmac(Lam[3], -0.14464285714285716, Ops::fmac(Lam[2], -0.14464285714285716, Ops::fmac(Lam[1], -0.14464285714285716, Ops::mulc(Lam[0], -0.14464285714285716))))));
    K[130] = Ops::fmac(Lam[8], 1.4464285714285714, Ops::fmac(Lam[7], -0.2892857142857143, Ops::fmac(Lam[3], 0.5785714285714286, Ops::fmac(Lam[2], 0.5785714285714286, Ops::mulc(Lam[0], 0.5785714285714286)))));
    K[131] = Ops::fmac(Lam[8], 0.7232142857142857, Ops::fmac(Lam[7], -0.14464285714285716, Ops::fmac(Lam[5], 0.7232142857142857, Ops::fmac(Lam[3], 0.5785714285714286, Ops::fmac(Lam[2], -0.14464285714285716, Ops::mulc(Lam[1], 0.5785714285714286))))));
    K[132] = Ops::fmac(Lam[9], 1.1571428571428573, Ops::fmac(Lam[3], 1.1571428571428573, Ops::mulc(Lam[0], 1.4464285714285714)));
    K[133] = Ops::fmac(Lam[9], -0.43392857142857144, Ops::fmac(Lam[3], 0.2892857142857143, Ops::mulc(Lam[0], -0.43392857142857144)));
    K[134] = Ops::fmac(Lam[8], -0.14464285714285716, Ops::fmac(Lam[6], -0.14464285714285716, Ops::fmac(Lam[2], -0.14464285714285716, Ops::mulc(Lam[1], -0.14464285714285716))));
    K[135] = Ops::fmac(Lam[8], -0.14464285714285716, Ops::fmac(Lam[6], -0.14464285714285716, Ops::fmac(Lam[2], -0.14464285714285716, Ops::mulc(Lam[1], -0.14464285714285716))));
    K[136] = Ops::fmac(Lam[9], -0.14464285714285716, Ops::fmac(Lam[6], -0.14464285714285716, Ops::fmac(Lam[3], -0.14464285714285716, Ops::mulc(Lam[1], -0.2892857142857143))));
    K[137] = Ops::fmac(Lam[9], -0.14464285714285716, Ops::fmac(Lam[6], -0.14464285714285716, Ops::fmac(Lam[3], -0.2892857142857143, Ops::mulc(Lam[1], -0.43392857142857144))));
    K[138] = Ops::fmac(Lam[9], -0.14464285714285716, Ops::fmac(Lam[8], -0.14464285714285716, Ops::fmac(Lam[3], -0.14464285714285716, Ops::mulc(Lam[2], -0.2892857142857143))));
    K[139] = Ops::fmac(Lam[9], -0.14464285714285716, Ops::fmac(Lam[8], -0.14464285714285716, Ops::fmac(Lam[3], -0.2892857142857143, Ops::mulc(Lam[2], -0.43392857142857144))));
    K[140] = Ops::fmac(Lam[8], 0.5785714285714286, Ops::fmac(Lam[6], 0.5785714285714286, Ops::fmac(Lam[3], -0.14464285714285716, Ops::fmac(Lam[2], 0.7232142857142857, Ops::fmac(Lam[1], 0.7232142857142857, Ops::mulc(Lam[0], -0.14464285714285716))))));
    K[141] = Ops::fmac(Lam[9], 0.5785714285714286, Ops::fmac(Lam[6], 0.5785714285714286, Ops::fmac(Lam[3], 0.5785714285714286, Ops::fmac(Lam[1], 1.4464285714285714, Ops::mulc(Lam[0], -0.2892857142857143)))));
    K[142] = Ops::fmac(Lam[9], 0.5785714285714286, Ops::fmac(Lam[8], 0.5785714285714286, Ops::fmac(Lam[3], 0.5785714285714286, Ops::fmac(Lam[2], 1.4464285714285714, Ops::mulc(Lam[0], -0.2892857142857143)))));
    K[143] = Ops::fmac(Lam[9], -0.14464285714285716, Ops::fmac(Lam[8], -0.14464285714285716, Ops::fmac(Lam[6], -0.14464285714285716, Ops::fmac(Lam[3], -0.14464285714285716, Ops::fmac(Lam[2], -0.2892857142857143, Ops::mulc(Lam[1], -0.2892857142857143))))));
    K[144] = Ops::fmac(Lam[9], 1.4464285714285714, Ops::fmac(Lam[3], 1.1571428571428573, Ops::mulc(Lam[0], 1.1571428571428573)));
    K[145] = Ops::fmac(Lam[8], -0.14464285714285716, Ops::fmac(Lam[6], -0.14464285714285716, Ops::fmac(Lam[2], -0.14464285714285716, Ops::mulc(Lam[1], -0.14464285714285716))));
    K[146] = Ops::fmac(Lam[8], -0.14464285714285716, Ops::fmac(Lam[6], -0.14464285714285716, Ops::fmac(Lam[2], -0.14464285714285716, Ops::mulc(Lam[1], -0.14464285714285716))));
    K[147] = Ops::fmac(Lam[9], -0.14464285714285716, Ops::fmac(Lam[6], -0.2892857142857143, Ops::fmac(Lam[3], -0.14464285714285716, Ops::mulc(Lam[1], -0.43392857142857144))));
    K[148] = Ops::fmac(Lam[9], 0.7232142857142857, Ops::fmac(Lam[6], 0.5785714285714286, Ops::fmac(Lam[3], 0.5785714285714286, Ops::mulc(Lam[1], 1.1571428571428573))));
    K[149] = Ops::fmac(Lam[9], -0.14464285714285716, Ops::fmac(Lam[8], -0.2892857142857143, Ops::fmac(Lam[3], -0.14464285714285716, Ops::mulc(Lam[2], -0.43392857142857144))));
    K[150] = Ops::fmac(Lam[9], 0.7232142857142857, Ops::fmac(Lam[8], 0.5785714285714286, Ops::fmac(Lam[3], 0.5785714285714286, Ops::mulc(Lam[2], 1.1571428571428573))));
    K[151] = Ops::fmac(Lam[8], -0.2892857142857143, Ops::fmac(Lam[6], -0.2892857142857143, Ops::fmac(Lam[3], -0.14464285714285716, Ops::fmac(Lam[2], -0.14464285714285716, Ops::fmac(Lam[1], -0.14464285714285716, Ops::mulc(Lam[0], -0.14464285714285716))))));
    K[152] = Ops::fmac(Lam[9], -0.2892857142857143, Ops::fmac(Lam[6], 1.4464285714285714, Ops::fmac(Lam[3], 0.5785714285714286, Ops::fmac(Lam[1], 0.5785714285714286, Ops::mulc(Lam[0], 0.5785714285714286)))));
    K[153] = Ops::fmac(Lam[9], -0.2892857142857143, Ops::fmac(Lam[8], 1.4464285714285714, Ops::fmac(Lam[3], 0.5785714285714286, Ops::fmac(Lam[2], 0.5785714285714286, Ops::mulc(Lam[0], 0.5785714285714286)))));
    K[154] = Ops::fmac(Lam[9], -0.14464285714285716, Ops::fmac(Lam[8], 0.7232142857142857, Ops::fmac(Lam[6], 0.7232142857142857, Ops::fmac(Lam[3], -0.14464285714285716, Ops::fmac(Lam[2], 0.5785714285714286, Ops::mulc(Lam[1], 0.5785714285714286))))));
    K[155] = Ops::fmac(Lam[7], 1.1571428571428573, Ops::fmac(Lam[5], 1.1571428571428573, Ops::mulc(Lam[4], 1.4464285714285714)));
    K[156] = Ops::fmac(Lam[7], -0.43392857142857144, Ops::fmac(Lam[5], 0.2892857142857143, Ops::mulc(Lam[4], -0.43392857142857144)));
    K[157] = Ops::fmac(Lam[8], 1.1571428571428573, Ops::fmac(Lam[6], 0.5785714285714286, Ops::fmac(Lam[5], 0.5785714285714286, Ops::mulc(Lam[4], 0.7232142857142857))));
    K[158] = Ops::fmac(Lam[8], -0.43392857142857144, Ops::fmac(Lam[6], -0.2892857142857143, Ops::fmac(Lam[5], -0.14464285714285716, Ops::mulc(Lam[4], -0.14464285714285716))));
    K[159] = Ops::fmac(Lam[8], -0.14464285714285716, Ops::fmac(Lam[7], -0.14464285714285716, Ops::fmac(Lam[6], -0.43392857142857144, Ops::mulc(Lam[5], -0.2892857142857143))));
    K[160] = Ops::fmac(Lam[8], -0.14464285714285716, Ops::fmac(Lam[7], -0.14464285714285716, Ops::fmac(Lam[6], -0.2892857142857143, Ops::mulc(Lam[5], -0.14464285714285716))));
    K[161] = Ops::fmac(Lam[7], 0.5785714285714286, Ops::fmac(Lam[5], 0.5785714285714286, Ops::fmac(Lam[4], -0.2892857142857143, Ops::fmac(Lam[2], 0.5785714285714286, Ops::mulc(Lam[1], 1.4464285714285714)))));
    K[162] = Ops::fmac(Lam[8], 0.5785714285714286, Ops::fmac(Lam[6], 0.7232142857142857, Ops::fmac(Lam[5], -0.14464285714285716, Ops::fmac(Lam[4], -0.14464285714285716, Ops::fmac(Lam[2], 0.5785714285714286, Ops::mulc(Lam[1], 0.7232142857142857))))));
    K[163] = Ops::fmac(Lam[8], -0.14464285714285716, Ops::fmac(Lam[7], -0.14464285714285716, Ops::fmac(Lam[6], -0.2892857142857143, Ops::fmac(Lam[5], -0.14464285714285716, Ops::fmac(Lam[2], -0.14464285714285716, Ops::mulc(Lam[1], -0.2892857142857143))))));
    K[164] = Ops::fmac(Lam[8], 0.5785714285714286, Ops::fmac(Lam[7], 0.5785714285714286, Ops::fmac(Lam[6], 1.4464285714285714, Ops::fmac(Lam[5], 0.5785714285714286, Ops::mulc(Lam[4], -0.2892857142857143)))));
    K[165] = Ops::fmac(Lam[7], 1.4464285714285714, Ops::fmac(Lam[5], 1.1571428571428573, Ops::mulc(Lam[4], 1.1571428571428573)));
    K[166] = Ops::fmac(Lam[8], -0.43392857142857144, Ops::fmac(Lam[6], -0.14464285714285716, Ops::fmac(Lam[5], -0.2892857142857143, Ops::mulc(Lam[4], -0.14464285714285716))));
    K[167] = Ops::fmac(Lam[8], -0.2892857142857143, Ops::fmac(Lam[6], -0.14464285714285716, Ops::fmac(Lam[5], -0.14464285714285716, Ops::mulc(Lam[4], -0.14464285714285716))));
    K[168] = Ops::fmac(Lam[8], 0.5785714285714286, Ops::fmac(Lam[7], 0.7232142857142857, Ops::fmac(Lam[6], 1.1571428571428573, Ops::mulc(Lam[5], 0.5785714285714286))));
    K[169] = Ops::fmac(Lam[8], -0.2892857142857143, Ops::fmac(Lam[7], -0.14464285714285716, Ops::fmac(Lam[6], -0.43392857142857144, Ops::mulc(Lam[5], -0.14464285714285716))));
    K[170] = Ops::fmac(Lam[7], -0.2892857142857143, Ops::fmac(Lam[5], 0.5785714285714286, Ops::fmac(Lam[4], 0.5785714285714286, Ops::fmac(Lam[2], 1.4464285714285714, Ops::mulc(Lam[1], 0.5785714285714286)))));
    K[171] = Ops::fmac(Lam[8], -0.2892857142857143, Ops::fmac(Lam[6], -0.14464285714285716, Ops::fmac(Lam[5], -0.14464285714285716, Ops::fmac(Lam[4], -0.14464285714285716, Ops::fmac(Lam[2], -0.2892857142857143, Ops::mulc(Lam[1], -0.14464285714285716))))));
    K[172] = Ops::fmac(Lam[8], 0.7232142857142857, Ops::fmac(Lam[7], -0.14464285714285716, Ops::fmac(Lam[6], 0.5785714285714286, Ops::fmac(Lam[5], -0.14464285714285716, Ops::fmac(Lam[2], 0.7232142857142857, Ops::mulc(Lam[1], 0.5785714285714286))))));
    K[173] = Ops::fmac(Lam[8], 1.4464285714285714, Ops::fmac(Lam[7], -0.2892857142857143, Ops::fmac(Lam[6], 0.5785714285714286, Ops::fmac(Lam[5], 0.5785714285714286, Ops::mulc(Lam[4], 0.5785714285714286)))));
    K[174] = Ops::fmac(Lam[9], 1.1571428571428573, Ops::fmac(Lam[6], 1.1571428571428573, Ops::mulc(Lam[4], 1.4464285714285714)));
    K[175] = Ops::fmac(Lam[9], -0.43392857142857144, Ops::fmac(Lam[6], 0.2892857142857143, Ops::mulc(Lam[4], -0.43392857142857144)));
    K[176] = Ops::fmac(Lam[9], -0.14464285714285716, Ops::fmac(Lam[8], -0.14464285714285716, Ops::fmac(Lam[6], -0.14464285714285716, Ops::mulc(Lam[5], -0.2892857142857143))));
    K[177] = Ops::fmac(Lam[9], -0.14464285714285716, Ops::fmac(Lam[8], -0.14464285714285716, Ops::fmac(Lam[6], -0.2892857142857143, Ops::mulc(Lam[5], -0.43392857142857144))));
    K[178] = Ops::fmac(Lam[8], 0.5785714285714286, Ops::fmac(Lam[6], -0.14464285714285716, Ops::fmac(Lam[5], 0.7232142857142857, Ops::fmac(Lam[4], -0.14464285714285716, Ops::fmac(Lam[3], 0.5785714285714286, Ops::mulc(Lam[1], 0.7232142857142857))))));
    K[179] = Ops::fmac(Lam[9], 0.5785714285714286, Ops::fmac(Lam[6], 0.5785714285714286, Ops::fmac(Lam[4], -0.2892857142857143, Ops::fmac(Lam[3], 0.5785714285714286, Ops::mulc(Lam[1], 1.4464285714285714)))));
    K[180] = Ops::fmac(Lam[9], -0.14464285714285716, Ops::fmac(Lam[8], -0.14464285714285716, Ops::fmac(Lam[6], -0.14464285714285716, Ops::fmac(Lam[5], -0.2892857142857143, Ops::fmac(Lam[3], -0.14464285714285716, Ops::mulc(Lam[1], -0.2892857142857143))))));
    K[181] = Ops::fmac(Lam[9], 0.5785714285714286, Ops::fmac(Lam[8], 0.5785714285714286, Ops::fmac(Lam[6], 0.5785714285714286, Ops::fmac(Lam[5], 1.4464285714285714, Ops::mulc(Lam[4], -0.2892857142857143)))));
    K[182] = Ops::fmac(Lam[9], 1.4464285714285714, Ops::fmac(Lam[6], 1.1571428571428573, Ops::mulc(Lam[4], 1.1571428571428573)));
    K[183] = Ops::fmac(Lam[9], -0.14464285714285716, Ops::fmac(Lam[8], -0.2892857142857143, Ops::fmac(Lam[6], -0.14464285714285716, Ops::mulc(Lam[5], -0.43392857142857144))));
    K[184] = Ops::fmac(Lam[9], 0.7232142857142857, Ops::fmac(Lam[8], 0.5785714285714286, Ops::fmac(Lam[6], 0.5785714285714286, Ops::mulc(Lam[5], 1.1571428571428573))));
    K[185] = Ops::fmac(Lam[8], -0.2892857142857143, Ops::fmac(Lam[6], -0.14464285714285716, Ops::fmac(Lam[5], -0.14464285714285716, Ops::fmac(Lam[4], -0.14464285714285716, Ops::fmac(Lam[3], -0.2892857142857143, Ops::mulc(Lam[1], -0.14464285714285716))))));
    K[186] = Ops::fmac(Lam[9], -0.2892857142857143, Ops::fmac(Lam[6], 0.5785714285714286, Ops::fmac(Lam[4], 0.5785714285714286, Ops::fmac(Lam[3], 1.4464285714285714, Ops::mulc(Lam[1], 0.5785714285714286)))));
    K[187] = Ops::fmac(Lam[9], -0.14464285714285716, Ops::fmac(Lam[8], 0.7232142857142857, Ops::fmac(Lam[6], -0.14464285714285716, Ops::fmac(Lam[5], 0.5785714285714286, Ops::fmac(Lam[3], 0.7232142857142857, Ops::mulc(Lam[1], 0.5785714285714286))))));
    K[188] = Ops::fmac(Lam[9], -0.2892857142857143, Ops::fmac(Lam[8], 1.4464285714285714, Ops::fmac(Lam[6], 0.5785714285714286, Ops::fmac(Lam[5], 0.5785714285714286, Ops::mulc(Lam[4], 0.5785714285714286)))));
    K[189] = Ops::fmac(Lam[9], 1.1571428571428573, Ops::fmac(Lam[8], 1.1571428571428573, Ops::mulc(Lam[7], 1.4464285714285714)));
    K[190] = Ops::fmac(Lam[9], -0.43392857142857144, Ops::fmac(Lam[8], 0.2892857142857143, Ops::mulc(Lam[7], -0.43392857142857144)));
    K[191] = Ops::fmac(Lam[8], -0.14464285714285716, Ops::fmac(Lam[7], -0.14464285714285716, Ops::fmac(Lam[6], 0.5785714285714286, Ops::fmac(Lam[5], 0.7232142857142857, Ops::fmac(Lam[3], 0.5785714285714286, Ops::mulc(Lam[2], 0.7232142857142857))))));
    K[192] = Ops::fmac(Lam[9], -0.14464285714285716, Ops::fmac(Lam[8], -0.14464285714285716, Ops::fmac(Lam[6], -0.14464285714285716, Ops::fmac(Lam[5], -0.2892857142857143, Ops::fmac(Lam[3], -0.14464285714285716, Ops::mulc(Lam[2], -0.2892857142857143))))));
    K[193] = Ops::fmac(Lam[9], 0.5785714285714286, Ops::fmac(Lam[8], 0.5785714285714286, Ops::fmac(Lam[7], -0.2892857142857143, Ops::fmac(Lam[3], 0.5785714285714286, Ops::mulc(Lam[2], 1.4464285714285714)))));
    K[194] = Ops::fmac(Lam[9], 0.5785714285714286, Ops::fmac(Lam[8], 0.5785714285714286, Ops::fmac(Lam[7], -0.2892857142857143, Ops::fmac(Lam[6], 0.5785714285714286, Ops::mulc(Lam[5], 1.4464285714285714)))));
    K[195] = Ops::fmac(Lam[9], 1.4464285714285714, Ops::fmac(Lam[8], 1.1571428571428573, Ops::mulc(Lam[7], 1.1571428571428573)));
    K[196] = Ops::fmac(Lam[8], -0.14464285714285716, Ops::fmac(Lam[7], -0.14464285714285716, Ops::fmac(Lam[6], -0.2892857142857143, Ops::fmac(Lam[5], -0.14464285714285716, Ops::fmac(Lam[3], -0.2892857142857143, Ops::mulc(Lam[2], -0.14464285714285716))))));
    K[197] = Ops::fmac(Lam[9], -0.14464285714285716, Ops::fmac(Lam[8], -0.14464285714285716, Ops::fmac(Lam[6], 0.7232142857142857, Ops::fmac(Lam[5], 0.5785714285714286, Ops::fmac(Lam[3], 0.7232142857142857, Ops::mulc(Lam[2], 0.5785714285714286))))));
    K[198] = Ops::fmac(Lam[9], -0.2892857142857143, Ops::fmac(Lam[8], 0.5785714285714286, Ops::fmac(Lam[7], 0.5785714285714286, Ops::fmac(Lam[3], 1.4464285714285714, Ops::mulc(Lam[2], 0.5785714285714286)))));
    K[199] = Ops::fmac(Lam[9], -0.2892857142857143, Ops::fmac(Lam[8], 0.5785714285714286, Ops::fmac(Lam[7], 0.5785714285714286, Ops::fmac(Lam[6], 1.4464285714285714, Ops::mulc(Lam[5], 0.5785714285714286)))));
    K[200] = Ops::fmac(Lam[7], 3.4714285714285715, Ops::fmac(Lam[5], 3.4714285714285715, Ops::fmac(Lam[4], 3.4714285714285715, Ops::fmac(Lam[2], 3.4714285714285715, Ops::fmac(Lam[1], 3.4714285714285715, Ops::mulc(Lam[0], 3.4714285714285715))))));
    K[201] = Ops::fmac(Lam[8], 3.4714285714285715, Ops::fmac(Lam[6], 1.7357142857142858, Ops::fmac(Lam[5], 1.7357142857142858, Ops::fmac(Lam[4], 1.7357142857142858, Ops::fmac(Lam[3], 1.7357142857142858, Ops::fmac(Lam[2], 1.7357142857142858, Ops::fmac(Lam[1], 1.7357142857142858, Ops::mulc(Lam[0], 1.7357142857142858))))))));
    K[202] = Ops::fmac(Lam[8], 1.7357142857142858, Ops::fmac(Lam[7], 1.7357142857142858, Ops::fmac(Lam[6], 3.4714285714285715, Ops::fmac(Lam[5], 1.7357142857142858, Ops::fmac(Lam[3], 1.7357142857142858, Ops::fmac(Lam[2], 1.7357142857142858, Ops::fmac(Lam[1], 1.7357142857142858, Ops::mulc(Lam[0], 1.7357142857142858))))))));
    K[203] = Ops::fmac(Lam[8], 1.7357142857142858, Ops::fmac(Lam[7], 1.7357142857142858, Ops::fmac(Lam[6], 1.7357142857142858, Ops::fmac(Lam[5], 1.7357142857142858, Ops::fmac(Lam[4], 1.7357142857142858, Ops::fmac(Lam[3], 3.4714285714285715, Ops::fmac(Lam[2], 1.7357142857142858, Ops::mulc(Lam[1], 1.7357142857142858))))))));
    K[204] = Ops::fmac(Lam[9], 3.4714285714285715, Ops::fmac(Lam[6], 3.4714285714285715, Ops::fmac(Lam[4], 3.4714285714285715, Ops::fmac(Lam[3], 3.4714285714285715, Ops::fmac(Lam[1], 3.4714285714285715, Ops::mulc(Lam[0], 3.4714285714285715))))));
    K[205] = Ops::fmac(Lam[9], 1.7357142857142858, Ops::fmac(Lam[8], 1.7357142857142858, Ops::fmac(Lam[6], 1.7357142857142858, Ops::fmac(Lam[5], 3.4714285714285715, Ops::fmac(Lam[3], 1.7357142857142858, Ops::fmac(Lam[2], 1.7357142857142858, Ops::fmac(Lam[1], 1.7357142857142858, Ops::mulc(Lam[0], 1.7357142857142858))))))));
    K[206] = Ops::fmac(Lam[9], 1.7357142857142858, Ops::fmac(Lam[8], 1.7357142857142858, Ops::fmac(Lam[6], 1.7357142857142858, Ops::fmac(Lam[5], 1.7357142857142858, Ops::fmac(Lam[4], 1.7357142857142858, Ops::fmac(Lam[3], 1.7357142857142858, Ops::fmac(Lam[2], 3.4714285714285715, Ops::mulc(Lam[1], 1.7357142857142858))))))));
    K[207] = Ops::fmac(Lam[9], 3.4714285714285715, Ops::fmac(Lam[8], 3.4714285714285715, Ops::fmac(Lam[7], 3.4714285714285715, Ops::fmac(Lam[3], 3.4714285714285715, Ops::fmac(Lam[2], 3.4714285714285715, Ops::mulc(Lam[0], 3.4714285714285715))))));
    K[208] = Ops::fmac(Lam[9], 1.7357142857142858, Ops::fmac(Lam[8], 1.7357142857142858, Ops::fmac(Lam[7], 1.7357142857142858, Ops::fmac(Lam[6], 1.7357142857142858, Ops::fmac(Lam[5], 1.7357142857142858, Ops::fmac(Lam[3], 1.7357142857142858, Ops::fmac(Lam[2], 1.7357142857142858, Ops::mulc(Lam[1], 3.4714285714285715))))))));
    K[209] = Ops::fmac(Lam[9], 3.4714285714285715, Ops::fmac(Lam[8], 3.4714285714285715, Ops::fmac(Lam[7], 3.4714285714285715, Ops::fmac(Lam[6], 3.4714285714285715, Ops::fmac(Lam[5], 3.4714285714285715, Ops::mulc(Lam[4], 3.4714285714285715))))));
  }
  template <class Ops> __device__ __forceinline__ static void mass_upper_add(const typename Ops::T& vol, typename Ops::T* K) {
    K[0] = Ops::fmac(vol, 0.0035714285714285713, K[0]);
    K[1] = Ops::fmac(vol, 0.0004464285714285714, K[1]);
    K[2] = Ops::fmac(vol, 0.0004464285714285714, K[2]);
    K[3] = Ops::fmac(vol, 0.0004464285714285714, K[3]);
    K[4] = Ops::fmac(vol, -0.0026785714285714286, K[4]);
    K[5] = Ops::fmac(vol, 0.0013392857142857143, K[5]);
    K[6] = Ops::fmac(vol, -0.0026785714285714286, K[6]);
    K[7] = Ops::fmac(vol, 0.0013392857142857143, K[7]);
    K[8] = Ops::fmac(vol, -0.0026785714285714286, K[8]);
    K[9] = Ops::fmac(vol, 0.0013392857142857143, K[9]);
    K[10] = Ops::fmac(vol, 0.0006696428571428571, K[10]);
    K[11] = Ops::fmac(vol, 0.0006696428571428571, K[11]);
    K[12] = Ops::fmac(vol, 0.0006696428571428571, K[12]);
    K[13] = Ops::fmac(vol, 0.0006696428571428571, K[13]);
    K[14] = Ops::fmac(vol, 0.0006696428571428571, K[14]);
    K[15] = Ops::fmac(vol, 0.0006696428571428571, K[15]);
    K[16] = Ops::fmac(vol, 0.0040178571428571425, K[16]);
    K[17] = Ops::fmac(vol, 0.0040178571428571425, K[17]);
    K[18] = Ops::fmac(vol, 0.0040178571428571425, K[18]);
    K[19] = Ops::fmac(vol, 0.008035714285714285, K[19]);
    K[20] = Ops::fmac(vol, 0.0035714285714285713, K[20]);
    K[21] = Ops::fmac(vol, 0.0004464285714285714, K[21]);
    K[22] = Ops::fmac(vol, 0.0004464285714285714, K[22]);
    K[23] = Ops::fmac(vol, 0.0013392857142857143, K[23]);
    K[24] = Ops::fmac(vol, -0.0026785714285714286, K[24]);
    K[25] = Ops::fmac(vol, 0.0006696428571428571, K[25]);
    K[26] = Ops::fmac(vol, 0.0006696428571428571, K[26]);
    K[27] = Ops::fmac(vol, 0.0006696428571428571, K[27]);
    K[28] = Ops::fmac(vol, 0.0006696428571428571, K[28]);
    K[29] = Ops::fmac(vol, -0.0026785714285714286, K[29]);
    K[30] = Ops::fmac(vol, 0.0013392857142857143, K[30]);
    K[31] = Ops::fmac(vol, -0.0026785714285714286, K[31]);
    K[32] = Ops::fmac(vol, 0.0013392857142857143, K[32]);
    K[33] = Ops::fmac(vol, 0.0006696428571428571, K[33]);
    K[34] = Ops::fmac(vol, 0.0006696428571428571, K[34]);
    K[35] = Ops::fmac(vol, 0.0040178571428571425, K[35]);
    K[36] = Ops::fmac(vol, 0.0040178571428571425, K[36]);
    K[37] = Ops::fmac(vol, 0.008035714285714285, K[37]);
    K[38] = Ops::fmac(vol, 0.0040178571428571425, K[38]);
    K[39] = Ops::fmac(vol, 0.0035714285714285713, K[39]);
    K[40] = Ops::fmac(vol, 0.0004464285714285714, K[40]);
    K[41] = Ops::fmac(vol, 0.0006696428571428571, K[41]);
    K[42] = Ops::fmac(vol, 0.0006696428571428571, K[42]);
    K[43] = Ops::fmac(vol, 0.0013392857142857143, K[43]);
    K[44] = Ops::fmac(vol, -0.0026785714285714286, K[44]);
    K[45] = Ops::fmac(vol, 0.0006696428571428571, K[45]);
    K[46] = Ops::fmac(vol, 0.0006696428571428571, K[46]);
    K[47] = Ops::fmac(vol, 0.0013392857142857143, K[47]);
    K[48] = Ops::fmac(vol, -0.0026785714285714286, K[48]);
    K[49] = Ops::fmac(vol, 0.0006696428571428571, K[49]);
    K[50] = Ops::fmac(vol, 0.0006696428571428571, K[50]);
    K[51] = Ops::fmac(vol, -0.0026785714285714286, K[51]);
    K[52] = Ops::fmac(vol, 0.0013392857142857143, K[52]);
    K[53] = Ops::fmac(vol, 0.0040178571428571425, K[53]);
    K[54] = Ops::fmac(vol, 0.008035714285714285, K[54]);
    K[55] = Ops::fmac(vol, 0.0040178571428571425, K[55]);
    K[56] = Ops::fmac(vol, 0.0040178571428571425, K[56]);
    K[57] = Ops::fmac(vol, 0.0035714285714285713, K[57]);
    K[58] = Ops::fmac(vol, 0.0006696428571428571, K[58]);
    K[59] = Ops::fmac(vol, 0.0006696428571428571, K[59]);
    K[60] = Ops::fmac(vol, 0.0006696428571428571, K[60]);
    K[61] = Ops::fmac(vol, 0.0006696428571428571, K[61]);
    K[62] = Ops::fmac(vol, 0.0013392857142857143, K[62]);
    K[63] = Ops::fmac(vol, -0.0026785714285714286, K[63]);
    K[64] = Ops::fmac(vol, 0.0006696428571428571, K[64]);
    K[65] = Ops::fmac(vol, 0.0006696428571428571, K[65]);
    K[66] = Ops::fmac(vol, 0.0013392857142857143, K[66]);
    K[67] = Ops::fmac(vol, -0.0026785714285714286, K[67]);
    K[68] = Ops::fmac(vol, 0.0013392857142857143, K[68]);
    K[69] = Ops::fmac(vol, -0.0026785714285714286, K[69]);
    K[70] = Ops::fmac(vol, 0.008035714285714285, K[70]);
    K[71] = Ops::fmac(vol, 0.0040178571428571425, K[71]);
    K[72] = Ops::fmac(vol, 0.0040178571428571425, K[72]);
    K[73] = Ops::fmac(vol, 0.0040178571428571425, K[73]);
    K[74] = Ops::fmac(vol, 0.024107142857142858, K[74]);
    K[75] = Ops::fmac(vol, -0.012053571428571429, K[75]);
    K[76] = Ops::fmac(vol, 0.012053571428571429, K[76]);
    K[77] = Ops::fmac(vol, -0.0060267857142857146, K[77]);
    K[78] = Ops::fmac(vol, 0.012053571428571429, K[78]);
    K[79] = Ops::fmac(vol, -0.0060267857142857146, K[79]);
    K[80] = Ops::fmac(vol, -0.0060267857142857146, K[80]);
    K[82] = Ops::fmac(vol, -0.0060267857142857146, K[82]);
    K[89] = Ops::fmac(vol, -0.012053571428571429, K[89]);
    K[90] = Ops::fmac(vol, 0.024107142857142858, K[90]);
    K[91] = Ops::fmac(vol, -0.0060267857142857146, K[91]);
    K[93] = Ops::fmac(vol, -0.0060267857142857146, K[93]);
    K[95] = Ops::fmac(vol, 0.012053571428571429, K[95]);
    K[96] = Ops::fmac(vol, -0.0060267857142857146, K[96]);
    K[97] = Ops::fmac(vol, 0.012053571428571429, K[97]);
    K[98] = Ops::fmac(vol, -0.0060267857142857146, K[98]);
    K[103] = Ops::fmac(vol, -0.012053571428571429, K[103]);
    K[105] = Ops::fmac(vol, 0.024107142857142858, K[105]);
    K[106] = Ops::fmac(vol, -0.012053571428571429, K[106]);
    K[107] = Ops::fmac(vol, 0.012053571428571429, K[107]);
    K[108] = Ops::fmac(vol, -0.0060267857142857146, K[108]);
    K[110] = Ops::fmac(vol, -0.0060267857142857146, K[110]);
    K[113] = Ops::fmac(vol, -0.0060267857142857146, K[113]);
    K[118] = Ops::fmac(vol, -0.012053571428571429, K[118]);
    K[119] = Ops::fmac(vol, 0.024107142857142858, K[119]);
    K[120] = Ops::fmac(vol, -0.0060267857142857146, K[120]);
    K[122] = Ops::fmac(vol, -0.0060267857142857146, K[122]);
    K[123] = Ops::fmac(vol, 0.012053571428571429, K[123]);
    K[126] = Ops::fmac(vol, 0.012053571428571429, K[126]);
    K[127] = Ops::fmac(vol, -0.0060267857142857146, K[127]);
    K[129] = Ops::fmac(vol, -0.012053571428571429, K[129]);
    K[132] = Ops::fmac(vol, 0.024107142857142858, K[132]);
    K[133] = Ops::fmac(vol, -0.012053571428571429, K[133]);
    K[137] = Ops::fmac(vol, -0.0060267857142857146, K[137]);
    K[139] = Ops::fmac(vol, -0.0060267857142857146, K[139]);
    K[143] = Ops::fmac(vol, -0.012053571428571429, K[143]);
    K[144] = Ops::fmac(vol, 0.024107142857142858, K[144]);
    K[147] = Ops::fmac(vol, -0.0060267857142857146, K[147]);
    K[148] = Ops::fmac(vol, 0.012053571428571429, K[148]);
    K[149] = Ops::fmac(vol, -0.0060267857142857146, K[149]);
    K[150] = Ops::fmac(vol, 0.012053571428571429, K[150]);
    K[151] = Ops::fmac(vol, -0.012053571428571429, K[151]);
    K[155] = Ops::fmac(vol, 0.024107142857142858, K[155]);
    K[156] = Ops::fmac(vol, -0.012053571428571429, K[156]);
    K[157] = Ops::fmac(vol, 0.012053571428571429, K[157]);
    K[158] = Ops::fmac(vol, -0.0060267857142857146, K[158]);
    K[159] = Ops::fmac(vol, -0.0060267857142857146, K[159]);
    K[163] = Ops::fmac(vol, -0.012053571428571429, K[163]);
    K[165] = Ops::fmac(vol, 0.024107142857142858, K[165]);
    K[166] = Ops::fmac(vol, -0.0060267857142857146, K[166]);
    K[168] = Ops::fmac(vol, 0.012053571428571429, K[168]);
    K[169] = Ops::fmac(vol, -0.0060267857142857146, K[169]);
    K[171] = Ops::fmac(vol, -0.012053571428571429, K[171]);
    K[174] = Ops::fmac(vol, 0.024107142857142858, K[174]);
    K[175] = Ops::fmac(vol, -0.012053571428571429, K[175]);
    K[177] = Ops::fmac(vol, -0.0060267857142857146, K[177]);
    K[180] = Ops::fmac(vol, -0.012053571428571429, K[180]);
    K[182] = Ops::fmac(vol, 0.024107142857142858, K[182]);
    K[183] = Ops::fmac(vol, -0.0060267857142857146, K[183]);
    K[184] = Ops::fmac(vol, 0.012053571428571429, K[184]);
    K[185] = Ops::fmac(vol, -0.012053571428571429, K[185]);
    K[189] = Ops::fmac(vol, 0.024107142857142858, K[189]);
    K[190] = Ops::fmac(vol, -0.012053571428571429, K[190]);
    K[192] = Ops::fmac(vol, -0.012053571428571429, K[192]);
    K[195] = Ops::fmac(vol, 0.024107142857142858, K[195]);
    K[196] = Ops::fmac(vol, -0.012053571428571429, K[196]);
    K[200] = Ops::fmac(vol, 0.09642857142857143, K[200]);
    K[201] = Ops::fmac(vol, 0.048214285714285716, K[201]);
    K[202] = Ops::fmac(vol, 0.048214285714285716, K[202]);
    K[203] = Ops::fmac(vol, 0.048214285714285716, K[203]);
    K[204] = Ops::fmac(vol, 0.09642857142857143, K[204]);
    K[205] = Ops::fmac(vol, 0.048214285714285716, K[205]);
    K[206] = Ops::fmac(vol, 0.048214285714285716, K[206]);
    K[207] = Ops::fmac(vol, 0.09642857142857143, K[207]);
    K[208] = Ops::fmac(vol, 0.048214285714285716, K[208]);
    K[209] = Ops::fmac(vol, 0.09642857142857143, K[209]);
  }
  template <class Ops> __device__ __forceinline__ static void mass_upper(const typename Ops::T& vol, typename Ops::T* K) {
    K[0] = Ops::mulc(vol, 0.0035714285714285713);
    K[1] = Ops::mulc(vol, 0.0004464285714285714);
    K[2] = Ops::mulc(vol, 0.0004464285714285714);
    K[3] = Ops::mulc(vol, 0.0004464285714285714);
    K[4] = Ops::mulc(vol, -0.0026785714285714286);
    K[5] = Ops::mulc(vol, 0.0013392857142857143);
    K[6] = Ops::mulc(vol, -0.0026785714285714286);
    K[7] = Ops::mulc(vol, 0.0013392857142857143);
    K[8] = Ops::mulc(vol, -0.0026785714285714286);
    K[9] = Ops::mulc(vol, 0.0013392857142857143);
    K[10] = Ops::mulc(vol, 0.0006696428571428571);
    K[11] = Ops::mulc(vol, 0.0006696428571428571);
    K[12] = Ops::mulc(vol, 0.0006696428571428571);
    K[13] = Ops::mulc(vol, 0.0006696428571428571);
    K[14] = Ops::mulc(vol, 0.0006696428571428571);
    K[15] = Ops::mulc(vol, 0.0006696428571428571);
    K[16] = Ops::mulc(vol, 0.0040178571428571425);
    K[17] = Ops::mulc(vol, 0.0040178571428571425);
    K[18] = Ops::mulc(vol, 0.0040178571428571425);
    K[19] = Ops::mulc(vol, 0.008035714285714285);
    K[20] = Ops::mulc(vol, 0.0035714285714285713);
    K[21] = Ops::mulc(vol, 0.0004464285714285714);
    K[22] = Ops::mulc(vol, 0.0004464285714285714);
    K[23] = Ops::mulc(vol, 0.0013392857142857143);
    K[24] = Ops::mulc(vol, -0.0026785714285714286);
    K[25] = Ops::mulc(vol, 0.0006696428571428571);
    K[26] = Ops::mulc(vol, 0.0006696428571428571);
    K[27] = Ops::mulc(vol, 0.0006696428571428571);
    K[28] = Ops::mulc(vol, 0.0006696428571428571);
    K[29] = Ops::mulc(vol, -0.0026785714285714286);
    K[30] = Ops::mulc(vol, 0.0013392857142857143);
    K[31] = Ops::mulc(vol, -0.0026785714285714286);
    K[32] = Ops::mulc(vol, 0.0013392857142857143);
    K[33] = Ops::mulc(vol, 0.0006696428571428571);
    K[34] = Ops::mulc(vol, 0.0006696428571428571);
    K[35] = Ops::mulc(vol, 0.0040178571428571425);
    K[36] = Ops::mulc(vol, 0.0040178571428571425);
    K[37] = Ops::mulc(vol, 0.008035714285714285);
    K[38] = Ops::mulc(vol, 0.0040178571428571425);
    K[39] = Ops::mulc(vol, 0.0035714285714285713);
    K[40] = Ops::mulc(vol, 0.0004464285714285714);
    K[41] = Ops::mulc(vol, 0.0006696428571428571);
    K[42] = Ops::mulc(vol, 0.0006696428571428571);
    K[43] = Ops::mulc(vol, 0.0013392857142857143);
    K[44] = Ops::mulc(vol, -0.0026785714285714286);
    K[45] = Ops::mulc(vol, 0.0006696428571428571);
    K[46] = Ops::mulc(vol, 0.0006696428571428571);
    K[47] = Ops::mulc(vol, 0.0013392857142857143);
    K[48] = Ops::mulc(vol, -0.0026785714285714286);
    K[49] = Ops::mulc(vol, 0.0006696428571428571);
    K[50] = Ops::mulc(vol, 0.0006696428571428571);
    K[51] = Ops::mulc(vol, -0.0026785714285714286);
    K[52] = Ops::mulc(vol, 0.0013392857142857143);
    K[53] = Ops::mulc(vol, 0.0040178571428571425);
    K[54] = Ops::mulc(vol, 0.008035714285714285);
    K[55] = Ops::mulc(vol, 0.0040178571428571425);
    K[56] = Ops::mulc(vol, 0.0040178571428571425);
    K[57] = Ops::mulc(vol, 0.0035714285714285713);
    K[58] = Ops::mulc(vol, 0.0006696428571428571);
    K[59] = Ops::mulc(vol, 0.0006696428571428571);
    K[60] = Ops::mulc(vol, 0.0006696428571428571);
    K[61] = Ops::mulc(vol, 0.0006696428571428571);
    K[62] = Ops::mulc(vol, 0.0013392857142857143);
    K[63] = Ops::mulc(vol, -0.0026785714285714286);
    K[64] = Ops::mulc(vol, 0.0006696428571428571);
    K[65] = Ops::mulc(vol, 0.0006696428571428571);
    K[66] = Ops::mulc(vol, 0.0013392857142857143);
    K[67] = Ops::mulc(vol, -0.0026785714285714286);
    K[68] = Ops::mulc(vol, 0.0013392857142857143);
    K[69] = Ops::mulc(vol, -0.0026785714285714286);
    K[70] = Ops::mulc(vol, 0.008035714285714285);
    K[71] = Ops::mulc(vol, 0.0040178571428571425);
    K[72] = Ops::mulc(vol, 0.0040178571428571425);
    K[73] = Ops::mulc(vol, 0.0040178571428571425);
    K[74] = Ops::mulc(vol, 0.024107142857142858);
    K[75] = Ops::mulc(vol, -0.012053571428571429);
    K[76] = Ops::mulc(vol, 0.012053571428571429);
    K[77] = Ops::mulc(vol, -0.0060267857142857146);
    K[78] = Ops::mulc(vol, 0.012053571428571429);
    K[79] = Ops::mulc(vol, -0.0060267857142857146);
    K[80] = Ops::mulc(vol, -0.0060267857142857146);
    K[81] = Ops::mulc(vol, 0.0);
    K[82] = Ops::mulc(vol, -0.0060267857142857146);
    K[83] = Ops::mulc(vol, 0.0);
    K[84] = Ops::mulc(vol, 0.0);
    K[85] = Ops::mulc(vol, 0.0);
    K[86] = Ops::mulc(vol, 0.0);
    K[87] = Ops::mulc(vol, 0.0);
    K[88] = Ops::mulc(vol, 0.0);
    K[89] = Ops::mulc(vol, -0.012053571428571429);
    K[90] = Ops::mulc(vol, 0.024107142857142858);
    K[91] = Ops::mulc(vol, -0.0060267857142857146);
    K[92] = Ops::mulc(vol, 0.0);
    K[93] = Ops::mulc(vol, -0.0060267857142857146);
    K[94] = Ops::mulc(vol, 0.0);
    K[95] = Ops::mulc(vol, 0.012053571428571429);
    K[96] = Ops::mulc(vol, -0.0060267857142857146);
    K[97] = Ops::mulc(vol, 0.012053571428571429);
    K[98] = Ops::mulc(vol, -0.0060267857142857146);
    K[99] = Ops::mulc(vol, 0.0);
    K[100] = Ops::mulc(vol, 0.0);
    K[101] = Ops::mulc(vol, 0.0);
    K[102] = Ops::mulc(vol, 0.0);
    K[103] = Ops::mulc(vol, -0.012053571428571429);
    K[104] = Ops::mulc(vol, 0.0);
    K[105] = Ops::mulc(vol, 0.024107142857142858);
    K[106] = Ops::mulc(vol, -0.012053571428571429);
    K[107] = Ops::mulc(vol, 0.012053571428571429);
    K[108] = Ops::mulc(vol, -0.0060267857142857146);
    K[109] = Ops::mulc(vol, 0.0);
    K[110] = Ops::mulc(vol, -0.0060267857142857146);
    K[111] = Ops::mulc(vol, 0.0);
    K[112] = Ops::mulc(vol, 0.0);
    K[113] = Ops::mulc(vol, -0.0060267857142857146);
    K[114] = Ops::mulc(vol, 0.0);
    K[115] = Ops::mulc(vol, 0.0);
    K[116] = Ops::mulc(vol, 0.0);
    K[117] = Ops::mulc(vol, 0.0);
    K[118] = Ops::mulc(vol, -0.012053571428571429);
    K[119] = Ops::mulc(vol, 0.024107142857142858);
    K[120] = Ops::mulc(vol, -0.0060267857142857146);
    K[121] = Ops::mulc(vol, 0.0);
    K[122] = Ops::mulc(vol, -0.0060267857142857146);
    K[123] = Ops::mulc(vol, 0.012053571428571429);
    K[124] = Ops::mulc(vol, 0.0);
    K[125] = Ops::mulc(vol, 0.0);
    K[126] = Ops::mulc(vol, 0.012053571428571429);
    K[127] = Ops::mulc(vol, -0.0060267857142857146);
    K[128] = Ops::mulc(vol, 0.0);
    K[129] = Ops::mulc(vol, -0.012053571428571429);
    K[130] = Ops::mulc(vol, 0.0);
    K[131] = Ops::mulc(vol, 0.0);
    K[132] = Ops::mulc(vol, 0.024107142857142858);
    K[133] = Ops::mulc(vol, -0.012053571428571429);
    K[134] = Ops::mulc(vol, 0.0);
    K[135] = Ops::mulc(vol, 0.0);
    K[136] = Ops::mulc(vol, 0.0);
    K[137] = Ops::mulc(vol, -0.0060267857142857146);
    K[138] = Ops::mulc(vol, 0.0);
    K[139] = Ops::mulc(vol, -0.0060267857142857146);
    K[140] = Ops::mulc(vol, 0.0);
    K[141] = Ops::mulc(vol, 0.0);
    K[142] = Ops::mulc(vol, 0.0);
    K[143] = Ops::mulc(vol, -0.012053571428571429);
    K[144] = Ops::mulc(vol, 0.024107142857142858);
    K[145] = Ops::mulc(vol, 0.0);
    K[146] = Ops::mulc(vol, 0.0);
    K[147] = Ops::mulc(vol, -0.0060267857142857146);
    K[148] = Ops::mulc(vol, 0.012053571428571429);
    K[149] = Ops::mulc(vol, -0.0060267857142857146);
    K[150] = Ops::mulc(vol, 0.012053571428571429);
    K[151] = Ops::mulc(vol, -0.012053571428571429);
    K[152] = Ops::mulc(vol, 0.0);
    K[153] = Ops::mulc(vol, 0.0);
    K[154] = Ops::mulc(vol, 0.0);
    K[155] = Ops::mulc(vol, 0.024107142857142858);
    K[156] = Ops::mulc(vol, -0.012053571428571429);
    K[157] = Ops::mulc(vol, 0.012053571428571429);
    K[158] = Ops::mulc(vol, -0.0060267857142857146);
    K[159] = Ops::mulc(vol, -0.0060267857142857146);
    K[160] = Ops::mulc(vol, 0.0);
    K[161] = Ops::mulc(vol, 0.0);
    K[162] = Ops::mulc(vol, 0.0);
    K[163] = Ops::mulc(vol, -0.012053571428571429);
    K[164] = Ops::mulc(vol, 0.0);
    K[165] = Ops::mulc(vol, 0.024107142857142858);
    K[166] = Ops::mulc(vol, -0.0060267857142857146);
    K[167] = Ops::mulc(vol, 0.0);
    K[168] = Ops::mulc(vol, 0.012053571428571429);
    K[169] = Ops::mulc(vol, -0.0060267857142857146);
    K[170] = Ops::mulc(vol, 0.0);
    K[171] = Ops::mulc(vol, -0.012053571428571429);
    K[172] = Ops::mulc(vol, 0.0);
    K[173] = Ops::mulc(vol, 0.0);
    K[174] = Ops::mulc(vol, 0.024107142857142858);
    K[175] = Ops::mulc(vol, -0.012053571428571429);
    K[176] = Ops::mulc(vol, 0.0);
    K[177] = Ops::mulc(vol, -0.0060267857142857146);
    K[178] = Ops::mulc(vol, 0.0);
    K[179] = Ops::mulc(vol, 0.0);
    K[180] = Ops::mulc(vol, -0.012053571428571429);
    K[181] = Ops::mulc(vol, 0.0);
    K[182] = Ops::mulc(vol, 0.024107142857142858);
    K[183] = Ops::mulc(vol, -0.0060267857142857146);
    K[184] = Ops::mulc(vol, 0.012053571428571429);
    K[185] = Ops::mulc(vol, -0.012053571428571429);
    K[186] = Ops::mulc(vol, 0.0);
    K[187] = Ops::mulc(vol, 0.0);
    K[188] = Ops::mulc(vol, 0.0);
    K[189] = Ops::mulc(vol, 0.024107142857142858);
    K[190] = Ops::mulc(vol, -0.012053571428571429);
    K[191] = Ops::mulc(vol, 0.0);
    K[192] = Ops::mulc(vol, -0.012053571428571429);
    K[193] = Ops::mulc(vol, 0.0);
    K[194] = Ops::mulc(vol, 0.0);
    K[195] = Ops::mulc(vol, 0.024107142857142858);
    K[196] = Ops::mulc(vol, -0.012053571428571429);
    K[197] = Ops::mulc(vol, 0.0);
    K[198] = Ops::mulc(vol, 0.0);
    K[199] = Ops::mulc(vol, 0.0);
    K[200] = Ops::mulc(vol, 0.09642857142857143);
    K[201] = Ops::mulc(vol, 0.048214285714285716);
    K[202] = Ops::mulc(vol, 0.048214285714285716);
    K[203] = Ops::mulc(vol, 0.048214285714285716);
    K[204] = Ops::mulc(vol, 0.09642857142857143);
    K[205] = Ops::mulc(vol, 0.048214285714285716);
    K[206] = Ops::mulc(vol, 0.048214285714285716);
    K[207] = Ops::mulc(vol, 0.09642857142857143);
    K[208] = Ops::mulc(vol, 0.048214285714285716);
    K[209] = Ops::mulc(vol, 0.09642857142857143);
  }
  template <class Ops, bool STIFF, bool MASS> __device__ __forceinline__ static void action_upper(const typename Ops::T* Lam, const typename Ops::T& vol, const typename Ops::T* x, typename Ops::T* y) {
    typename Ops::T k;
    { if constexpr (STIFF) { k = Ops::mulc(Lam[0], 0.35714285714285715); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, 0.0035714285714285713, k); } y[0] = Ops::fma3(k, x[0], y[0]); }
    { if constexpr (STIFF) { k = Ops::mulc(Lam[1], 0.06785714285714285); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, 0.0004464285714285714, k); } y[0] = Ops::fma3(k, x[1], y[0]); y[1] = Ops::fma3(k, x[0], y[1]); }
    { if constexpr (STIFF) { k = Ops::mulc(Lam[2], 0.06785714285714285); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, 0.0004464285714285714, k); } y[0] = Ops::fma3(k, x[2], y[0]); y[2] = Ops::fma3(k, x[0], y[2]); }
    { if constexpr (STIFF) { k = Ops::mulc(Lam[3], 0.06785714285714285); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, 0.0004464285714285714, k); } y[0] = Ops::fma3(k, x[3], y[0]); y[3] = Ops::fma3(k, x[0], y[3]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[1], 0.36964285714285716, Ops::mulc(Lam[0], -0.20892857142857144)); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, -0.0026785714285714286, k); } y[0] = Ops::fma3(k, x[4], y[0]); y[4] = Ops::fma3(k, x[0], y[4]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[1], -0.20892857142857144, Ops::mulc(Lam[0], 0.08035714285714286)); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, 0.0013392857142857143, k); } y[0] = Ops::fma3(k, x[5], y[0]); y[5] = Ops::fma3(k, x[0], y[5]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[2], 0.36964285714285716, Ops::mulc(Lam[0], -0.20892857142857144)); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, -0.0026785714285714286, k); } y[0] = Ops::fma3(k, x[6], y[0]); y[6] = Ops::fma3(k, x[0], y[6]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[2], -0.20892857142857144, Ops::mulc(Lam[0], 0.08035714285714286)); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, 0.0013392857142857143, k); } y[0] = Ops::fma3(k, x[7], y[0]); y[7] = Ops::fma3(k, x[0], y[7]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[3], 0.36964285714285716, Ops::mulc(Lam[0], -0.20892857142857144)); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, -0.0026785714285714286, k); } y[0] = Ops::fma3(k, x[8], y[0]); y[8] = Ops::fma3(k, x[0], y[8]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[3], -0.20892857142857144, Ops::mulc(Lam[0], 0.08035714285714286)); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, 0.0013392857142857143, k); } y[0] = Ops::fma3(k, x[9], y[0]); y[9] = Ops::fma3(k, x[0], y[9]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[2], 0.08035714285714286, Ops::mulc(Lam[1], 0.08035714285714286)); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, 0.0006696428571428571, k); } y[0] = Ops::fma3(k, x[10], y[0]); y[10] = Ops::fma3(k, x[0], y[10]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[2], 0.08035714285714286, Ops::mulc(Lam[1], 0.08035714285714286)); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, 0.0006696428571428571, k); } y[0] = Ops::fma3(k, x[11], y[0]); y[11] = Ops::fma3(k, x[0], y[11]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[3], 0.08035714285714286, Ops::mulc(Lam[1], 0.08035714285714286)); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, 0.0006696428571428571, k); } y[0] = Ops::fma3(k, x[12], y[0]); y[12] = Ops::fma3(k, x[0], y[12]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[3], 0.08035714285714286, Ops::mulc(Lam[1], 0.08035714285714286)); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, 0.0006696428571428571, k); } y[0] = Ops::fma3(k, x[13], y[0]); y[13] = Ops::fma3(k, x[0], y[13]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[3], 0.08035714285714286, Ops::mulc(Lam[2], 0.08035714285714286)); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, 0.0006696428571428571, k); } y[0] = Ops::fma3(k, x[14], y[0]); y[14] = Ops::fma3(k, x[0], y[14]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[3], 0.08035714285714286, Ops::mulc(Lam[2], 0.08035714285714286)); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, 0.0006696428571428571, k); } y[0] = Ops::fma3(k, x[15], y[0]); y[15] = Ops::fma3(k, x[0], y[15]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[2], -0.09642857142857143, Ops::fmac(Lam[1], -0.09642857142857143, Ops::mulc(Lam[0], 0.19285714285714287))); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, 0.0040178571428571425, k); } y[0] = Ops::fma3(k, x[16], y[0]); y[16] = Ops::fma3(k, x[0], y[16]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[3], -0.09642857142857143, Ops::fmac(Lam[1], -0.09642857142857143, Ops::mulc(Lam[0], 0.19285714285714287))); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, 0.0040178571428571425, k); } y[0] = Ops::fma3(k, x[17], y[0]); y[17] = Ops::fma3(k, x[0], y[17]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[3], -0.09642857142857143, Ops::fmac(Lam[2], -0.09642857142857143, Ops::mulc(Lam[0], 0.19285714285714287))); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, 0.0040178571428571425, k); } y[0] = Ops::fma3(k, x[18], y[0]); y[18] = Ops::fma3(k, x[0], y[18]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[3], 0.19285714285714287, Ops::fmac(Lam[2], 0.19285714285714287, Ops::mulc(Lam[1], 0.19285714285714287))); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, 0.008035714285714285, k); } y[0] = Ops::fma3(k, x[19], y[0]); y[19] = Ops::fma3(k, x[0], y[19]); }
    { if constexpr (STIFF) { k = Ops::mulc(Lam[4], 0.35714285714285715); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, 0.0035714285714285713, k); } y[1] = Ops::fma3(k, x[1], y[1]); }
    { if constexpr (STIFF) { k = Ops::mulc(Lam[5], 0.06785714285714285); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, 0.0004464285714285714, k); } y[1] = Ops::fma3(k, x[2], y[1]); y[2] = Ops::fma3(k, x[1], y[2]); }
    { if constexpr (STIFF) { k = Ops::mulc(Lam[6], 0.06785714285714285); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, 0.0004464285714285714, k); } y[1] = Ops::fma3(k, x[3], y[1]); y[3] = Ops::fma3(k, x[1], y[3]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[4], 0.08035714285714286, Ops::mulc(Lam[1], -0.20892857142857144)); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, 0.0013392857142857143, k); } y[1] = Ops::fma3(k, x[4], y[1]); y[4] = Ops::fma3(k, x[1], y[4]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[4], -0.20892857142857144, Ops::mulc(Lam[1], 0.36964285714285716)); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, -0.0026785714285714286, k); } y[1] = Ops::fma3(k, x[5], y[1]); y[5] = Ops::fma3(k, x[1], y[5]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[5], 0.08035714285714286, Ops::mulc(Lam[1], 0.08035714285714286)); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, 0.0006696428571428571, k); } y[1] = Ops::fma3(k, x[6], y[1]); y[6] = Ops::fma3(k, x[1], y[6]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[5], 0.08035714285714286, Ops::mulc(Lam[1], 0.08035714285714286)); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, 0.0006696428571428571, k); } y[1] = Ops::fma3(k, x[7], y[1]); y[7] = Ops::fma3(k, x[1], y[7]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[6], 0.08035714285714286, Ops::mulc(Lam[1], 0.08035714285714286)); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, 0.0006696428571428571, k); } y[1] = Ops::fma3(k, x[8], y[1]); y[8] = Ops::fma3(k, x[1], y[8]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[6], 0.08035714285714286, Ops::mulc(Lam[1], 0.08035714285714286)); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, 0.0006696428571428571, k); } y[1] = Ops::fma3(k, x[9], y[1]); y[9] = Ops::fma3(k, x[1], y[9]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[5], 0.36964285714285716, Ops::mulc(Lam[4], -0.20892857142857144)); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, -0.0026785714285714286, k); } y[1] = Ops::fma3(k, x[10], y[1]); y[10] = Ops::fma3(k, x[1], y[10]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[5], -0.20892857142857144, Ops::mulc(Lam[4], 0.08035714285714286)); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, 0.0013392857142857143, k); } y[1] = Ops::fma3(k, x[11], y[1]); y[11] = Ops::fma3(k, x[1], y[11]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[6], 0.36964285714285716, Ops::mulc(Lam[4], -0.20892857142857144)); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, -0.0026785714285714286, k); } y[1] = Ops::fma3(k, x[12], y[1]); y[12] = Ops::fma3(k, x[1], y[12]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[6], -0.20892857142857144, Ops::mulc(Lam[4], 0.08035714285714286)); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, 0.0013392857142857143, k); } y[1] = Ops::fma3(k, x[13], y[1]); y[13] = Ops::fma3(k, x[1], y[13]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[6], 0.08035714285714286, Ops::mulc(Lam[5], 0.08035714285714286)); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, 0.0006696428571428571, k); } y[1] = Ops::fma3(k, x[14], y[1]); y[14] = Ops::fma3(k, x[1], y[14]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[6], 0.08035714285714286, Ops::mulc(Lam[5], 0.08035714285714286)); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, 0.0006696428571428571, k); } y[1] = Ops::fma3(k, x[15], y[1]); y[15] = Ops::fma3(k, x[1], y[15]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[5], -0.09642857142857143, Ops::fmac(Lam[4], 0.19285714285714287, Ops::mulc(Lam[1], -0.09642857142857143))); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, 0.0040178571428571425, k); } y[1] = Ops::fma3(k, x[16], y[1]); y[16] = Ops::fma3(k, x[1], y[16]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[6], -0.09642857142857143, Ops::fmac(Lam[4], 0.19285714285714287, Ops::mulc(Lam[1], -0.09642857142857143))); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, 0.0040178571428571425, k); } y[1] = Ops::fma3(k, x[17], y[1]); y[17] = Ops::fma3(k, x[1], y[17]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[6], 0.19285714285714287, Ops::fmac(Lam[5], 0.19285714285714287, Ops::mulc(Lam[1], 0.19285714285714287))); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, 0.008035714285714285, k); } y[1] = Ops::fma3(k, x[18], y[1]); y[18] = Ops::fma3(k, x[1], y[18]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[6], -0.09642857142857143, Ops::fmac(Lam[5], -0.09642857142857143, Ops::mulc(Lam[4], 0.19285714285714287))); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, 0.0040178571428571425, k); } y[1] = Ops::fma3(k, x[19], y[1]); y[19] = Ops::fma3(k, x[1], y[19]); }
    { if constexpr (STIFF) { k = Ops::mulc(Lam[7], 0.35714285714285715); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, 0.0035714285714285713, k); } y[2] = Ops::fma3(k, x[2], y[2]); }
    { if constexpr (STIFF) { k = Ops::mulc(Lam[8], 0.06785714285714285); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, 0.0004464285714285714, k); } y[2] = Ops::fma3(k, x[3], y[2]); y[3] = Ops::fma3(k, x[2], y[3]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[5], 0.08035714285714286, Ops::mulc(Lam[2], 0.08035714285714286)); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, 0.0006696428571428571, k); } y[2] = Ops::fma3(k, x[4], y[2]); y[4] = Ops::fma3(k, x[2], y[4]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[5], 0.08035714285714286, Ops::mulc(Lam[2], 0.08035714285714286)); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, 0.0006696428571428571, k); } y[2] = Ops::fma3(k, x[5], y[2]); y[5] = Ops::fma3(k, x[2], y[5]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[7], 0.08035714285714286, Ops::mulc(Lam[2], -0.20892857142857144)); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, 0.0013392857142857143, k); } y[2] = Ops::fma3(k, x[6], y[2]); y[6] = Ops::fma3(k, x[2], y[6]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[7], -0.20892857142857144, Ops::mulc(Lam[2], 0.36964285714285716)); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, -0.0026785714285714286, k); } y[2] = Ops::fma3(k, x[7], y[2]); y[7] = Ops::fma3(k, x[2], y[7]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[8], 0.08035714285714286, Ops::mulc(Lam[2], 0.08035714285714286)); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, 0.0006696428571428571, k); } y[2] = Ops::fma3(k, x[8], y[2]); y[8] = Ops::fma3(k, x[2], y[8]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[8], 0.08035714285714286, Ops::mulc(Lam[2], 0.08035714285714286)); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, 0.0006696428571428571, k); } y[2] = Ops::fma3(k, x[9], y[2]); y[9] = Ops::fma3(k, x[2], y[9]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[7], 0.08035714285714286, Ops::mulc(Lam[5], -0.20892857142857144)); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, 0.0013392857142857143, k); } y[2] = Ops::fma3(k, x[10], y[2]); y[10] = Ops::fma3(k, x[2], y[10]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[7], -0.20892857142857144, Ops::mulc(Lam[5], 0.36964285714285716)); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, -0.0026785714285714286, k); } y[2] = Ops::fma3(k, x[11], y[2]); y[11] = Ops::fma3(k, x[2], y[11]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[8], 0.08035714285714286, Ops::mulc(Lam[5], 0.08035714285714286)); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, 0.0006696428571428571, k); } y[2] = Ops::fma3(k, x[12], y[2]); y[12] = Ops::fma3(k, x[2], y[12]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[8], 0.08035714285714286, Ops::mulc(Lam[5], 0.08035714285714286)); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, 0.0006696428571428571, k); } y[2] = Ops::fma3(k, x[13], y[2]); y[13] = Ops::fma3(k, x[2], y[13]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[8], 0.36964285714285716, Ops::mulc(Lam[7], -0.20892857142857144)); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, -0.0026785714285714286, k); } y[2] = Ops::fma3(k, x[14], y[2]); y[14] = Ops::fma3(k, x[2], y[14]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[8], -0.20892857142857144, Ops::mulc(Lam[7], 0.08035714285714286)); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, 0.0013392857142857143, k); } y[2] = Ops::fma3(k, x[15], y[2]); y[15] = Ops::fma3(k, x[2], y[15]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[7], 0.19285714285714287, Ops::fmac(Lam[5], -0.09642857142857143, Ops::mulc(Lam[2], -0.09642857142857143))); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, 0.0040178571428571425, k); } y[2] = Ops::fma3(k, x[16], y[2]); y[16] = Ops::fma3(k, x[2], y[16]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[8], 0.19285714285714287, Ops::fmac(Lam[5], 0.19285714285714287, Ops::mulc(Lam[2], 0.19285714285714287))); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, 0.008035714285714285, k); } y[2] = Ops::fma3(k, x[17], y[2]); y[17] = Ops::fma3(k, x[2], y[17]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[8], -0.09642857142857143, Ops::fmac(Lam[7], 0.19285714285714287, Ops::mulc(Lam[2], -0.09642857142857143))); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, 0.0040178571428571425, k); } y[2] = Ops::fma3(k, x[18], y[2]); y[18] = Ops::fma3(k, x[2], y[18]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[8], -0.09642857142857143, Ops::fmac(Lam[7], 0.19285714285714287, Ops::mulc(Lam[5], -0.09642857142857143))); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, 0.0040178571428571425, k); } y[2] = Ops::fma3(k, x[19], y[2]); y[19] = Ops::fma3(k, x[2], y[19]); }
    { if constexpr (STIFF) { k = Ops::mulc(Lam[9], 0.35714285714285715); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, 0.0035714285714285713, k); } y[3] = Ops::fma3(k, x[3], y[3]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[6], 0.08035714285714286, Ops::mulc(Lam[3], 0.08035714285714286)); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, 0.0006696428571428571, k); } y[3] = Ops::fma3(k, x[4], y[3]); y[4] = Ops::fma3(k, x[3], y[4]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[6], 0.08035714285714286, Ops::mulc(Lam[3], 0.08035714285714286)); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, 0.0006696428571428571, k); } y[3] = Ops::fma3(k, x[5], y[3]); y[5] = Ops::fma3(k, x[3], y[5]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[8], 0.08035714285714286, Ops::mulc(Lam[3], 0.08035714285714286)); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, 0.0006696428571428571, k); } y[3] = Ops::fma3(k, x[6], y[3]); y[6] = Ops::fma3(k, x[3], y[6]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[8], 0.08035714285714286, Ops::mulc(Lam[3], 0.08035714285714286)); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, 0.0006696428571428571, k); } y[3] = Ops::fma3(k, x[7], y[3]); y[7] = Ops::fma3(k, x[3], y[7]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[9], 0.08035714285714286, Ops::mulc(Lam[3], -0.20892857142857144)); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, 0.0013392857142857143, k); } y[3] = Ops::fma3(k, x[8], y[3]); y[8] = Ops::fma3(k, x[3], y[8]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[9], -0.20892857142857144, Ops::mulc(Lam[3], 0.36964285714285716)); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, -0.0026785714285714286, k); } y[3] = Ops::fma3(k, x[9], y[3]); y[9] = Ops::fma3(k, x[3], y[9]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[8], 0.08035714285714286, Ops::mulc(Lam[6], 0.08035714285714286)); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, 0.0006696428571428571, k); } y[3] = Ops::fma3(k, x[10], y[3]); y[10] = Ops::fma3(k, x[3], y[10]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[8], 0.08035714285714286, Ops::mulc(Lam[6], 0.08035714285714286)); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, 0.0006696428571428571, k); } y[3] = Ops::fma3(k, x[11], y[3]); y[11] = Ops::fma3(k, x[3], y[11]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[9], 0.08035714285714286, Ops::mulc(Lam[6], -0.20892857142857144)); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, 0.0013392857142857143, k); } y[3] = Ops::fma3(k, x[12], y[3]); y[12] = Ops::fma3(k, x[3], y[12]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[9], -0.20892857142857144, Ops::mulc(Lam[6], 0.36964285714285716)); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, -0.0026785714285714286, k); } y[3] = Ops::fma3(k, x[13], y[3]); y[13] = Ops::fma3(k, x[3], y[13]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[9], 0.08035714285714286, Ops::mulc(Lam[8], -0.20892857142857144)); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, 0.0013392857142857143, k); } y[3] = Ops::fma3(k, x[14], y[3]); y[14] = Ops::fma3(k, x[3], y[14]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[9], -0.20892857142857144, Ops::mulc(Lam[8], 0.36964285714285716)); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, -0.0026785714285714286, k); } y[3] = Ops::fma3(k, x[15], y[3]); y[15] = Ops::fma3(k, x[3], y[15]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[8], 0.19285714285714287, Ops::fmac(Lam[6], 0.19285714285714287, Ops::mulc(Lam[3], 0.19285714285714287))); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, 0.008035714285714285, k); } y[3] = Ops::fma3(k, x[16], y[3]); y[16] = Ops::fma3(k, x[3], y[16]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[9], 0.19285714285714287, Ops::fmac(Lam[6], -0.09642857142857143, Ops::mulc(Lam[3], -0.09642857142857143))); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, 0.0040178571428571425, k); } y[3] = Ops::fma3(k, x[17], y[3]); y[17] = Ops::fma3(k, x[3], y[17]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[9], 0.19285714285714287, Ops::fmac(Lam[8], -0.09642857142857143, Ops::mulc(Lam[3], -0.09642857142857143))); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, 0.0040178571428571425, k); } y[3] = Ops::fma3(k, x[18], y[3]); y[18] = Ops::fma3(k, x[3], y[18]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[9], 0.19285714285714287, Ops::fmac(Lam[8], -0.09642857142857143, Ops::mulc(Lam[6], -0.09642857142857143))); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, 0.0040178571428571425, k); } y[3] = Ops::fma3(k, x[19], y[3]); y[19] = Ops::fma3(k, x[3], y[19]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[4], 1.1571428571428573, Ops::fmac(Lam[1], 1.1571428571428573, Ops::mulc(Lam[0], 1.4464285714285714))); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, 0.024107142857142858, k); } y[4] = Ops::fma3(k, x[4], y[4]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[4], -0.43392857142857144, Ops::fmac(Lam[1], 0.2892857142857143, Ops::mulc(Lam[0], -0.43392857142857144))); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, -0.012053571428571429, k); } y[4] = Ops::fma3(k, x[5], y[4]); y[5] = Ops::fma3(k, x[4], y[5]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[5], 1.1571428571428573, Ops::fmac(Lam[2], 0.5785714285714286, Ops::fmac(Lam[1], 0.5785714285714286, Ops::mulc(Lam[0], 0.7232142857142857)))); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, 0.012053571428571429, k); } y[4] = Ops::fma3(k, x[6], y[4]); y[6] = Ops::fma3(k, x[4], y[6]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[5], -0.43392857142857144, Ops::fmac(Lam[2], -0.2892857142857143, Ops::fmac(Lam[1], -0.14464285714285716, Ops::mulc(Lam[0], -0.14464285714285716)))); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, -0.0060267857142857146, k); } y[4] = Ops::fma3(k, x[7], y[4]); y[7] = Ops::fma3(k, x[4], y[7]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[6], 1.1571428571428573, Ops::fmac(Lam[3], 0.5785714285714286, Ops::fmac(Lam[1], 0.5785714285714286, Ops::mulc(Lam[0], 0.7232142857142857)))); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, 0.012053571428571429, k); } y[4] = Ops::fma3(k, x[8], y[4]); y[8] = Ops::fma3(k, x[4], y[8]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[6], -0.43392857142857144, Ops::fmac(Lam[3], -0.2892857142857143, Ops::fmac(Lam[1], -0.14464285714285716, Ops::mulc(Lam[0], -0.14464285714285716)))); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, -0.0060267857142857146, k); } y[4] = Ops::fma3(k, x[9], y[4]); y[9] = Ops::fma3(k, x[4], y[9]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[5], -0.14464285714285716, Ops::fmac(Lam[4], -0.14464285714285716, Ops::fmac(Lam[2], -0.43392857142857144, Ops::mulc(Lam[1], -0.2892857142857143)))); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, -0.0060267857142857146, k); } y[4] = Ops::fma3(k, x[10], y[4]); y[10] = Ops::fma3(k, x[4], y[10]); }
    if constexpr (STIFF) { if constexpr (STIFF) { k = Ops::fmac(Lam[5], -0.14464285714285716, Ops::fmac(Lam[4], -0.14464285714285716, Ops::fmac(Lam[2], -0.2892857142857143, Ops::mulc(Lam[1], -0.14464285714285716)))); } else { k = Ops::zero(); } y[4] = Ops::fma3(k, x[11], y[4]); y[11] = Ops::fma3(k, x[4], y[11]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[6], -0.14464285714285716, Ops::fmac(Lam[4], -0.14464285714285716, Ops::fmac(Lam[3], -0.43392857142857144, Ops::mulc(Lam[1], -0.2892857142857143)))); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, -0.0060267857142857146, k); } y[4] = Ops::fma3(k, x[12], y[4]); y[12] = Ops::fma3(k, x[4], y[12]); }
    if constexpr (STIFF) { if constexpr (STIFF) { k = Ops::fmac(Lam[6], -0.14464285714285716, Ops::fmac(Lam[4], -0.14464285714285716, Ops::fmac(Lam[3], -0.2892857142857143, Ops::mulc(Lam[1], -0.14464285714285716)))); } else { k = Ops::zero(); } y[4] = Ops::fma3(k, x[13], y[4]); y[13] = Ops::fma3(k, x[4], y[13]); }
    if constexpr (STIFF) { if constexpr (STIFF) { k = Ops::fmac(Lam[6], -0.14464285714285716, Ops::fmac(Lam[5], -0.14464285714285716, Ops::fmac(Lam[3], -0.14464285714285716, Ops::mulc(Lam[2], -0.14464285714285716)))); } else { k = Ops::zero(); } y[4] = Ops::fma3(k, x[14], y[4]); y[14] = Ops::fma3(k, x[4], y[14]); }
    if constexpr (STIFF) { if constexpr (STIFF) { k = Ops::fmac(Lam[6], -0.14464285714285716, Ops::fmac(Lam[5], -0.14464285714285716, Ops::fmac(Lam[3], -0.14464285714285716, Ops::mulc(Lam[2], -0.14464285714285716)))); } else { k = Ops::zero(); } y[4] = Ops::fma3(k, x[15], y[4]); y[15] = Ops::fma3(k, x[4], y[15]); }
    if constexpr (STIFF) { if constexpr (STIFF) { k = Ops::fmac(Lam[5], 0.5785714285714286, Ops::fmac(Lam[4], 0.5785714285714286, Ops::fmac(Lam[2], 1.4464285714285714, Ops::fmac(Lam[1], 0.5785714285714286, Ops::mulc(Lam[0], -0.2892857142857143))))); } else { k = Ops::zero(); } y[4] = Ops::fma3(k, x[16], y[4]); y[16] = Ops::fma3(k, x[4], y[16]); }
    if constexpr (STIFF) { if constexpr (STIFF) { k = Ops::fmac(Lam[6], 0.5785714285714286, Ops::fmac(Lam[4], 0.5785714285714286, Ops::fmac(Lam[3], 1.4464285714285714, Ops::fmac(Lam[1], 0.5785714285714286, Ops::mulc(Lam[0], -0.2892857142857143))))); } else { k = Ops::zero(); } y[4] = Ops::fma3(k, x[17], y[4]); y[17] = Ops::fma3(k, x[4], y[17]); }
    if constexpr (STIFF) { if constexpr (STIFF) { k = Ops::fmac(Lam[6], 0.5785714285714286, Ops::fmac(Lam[5], 0.5785714285714286, Ops::fmac(Lam[3], 0.7232142857142857, Ops::fmac(Lam[2], 0.7232142857142857, Ops::fmac(Lam[1], -0.14464285714285716, Ops::mulc(Lam[0], -0.14464285714285716)))))); } else { k = Ops::zero(); } y[4] = Ops::fma3(k, x[18], y[4]); y[18] = Ops::fma3(k, x[4], y[18]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[6], -0.14464285714285716, Ops::fmac(Lam[5], -0.14464285714285716, Ops::fmac(Lam[4], -0.14464285714285716, Ops::fmac(Lam[3], -0.2892857142857143, Ops::fmac(Lam[2], -0.2892857142857143, Ops::mulc(Lam[1], -0.14464285714285716)))))); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, -0.012053571428571429, k); } y[4] = Ops::fma3(k, x[19], y[4]); y[19] = Ops::fma3(k, x[4], y[19]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[4], 1.4464285714285714, Ops::fmac(Lam[1], 1.1571428571428573, Ops::mulc(Lam[0], 1.1571428571428573))); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, 0.024107142857142858, k); } y[5] = Ops::fma3(k, x[5], y[5]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[5], -0.43392857142857144, Ops::fmac(Lam[2], -0.14464285714285716, Ops::fmac(Lam[1], -0.2892857142857143, Ops::mulc(Lam[0], -0.14464285714285716)))); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, -0.0060267857142857146, k); } y[5] = Ops::fma3(k, x[6], y[5]); y[6] = Ops::fma3(k, x[5], y[6]); }
    if constexpr (STIFF) { if constexpr (STIFF) { k = Ops::fmac(Lam[5], -0.2892857142857143, Ops::fmac(Lam[2], -0.14464285714285716, Ops::fmac(Lam[1], -0.14464285714285716, Ops::mulc(Lam[0], -0.14464285714285716)))); } else { k = Ops::zero(); } y[5] = Ops::fma3(k, x[7], y[5]); y[7] = Ops::fma3(k, x[5], y[7]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[6], -0.43392857142857144, Ops::fmac(Lam[3], -0.14464285714285716, Ops::fmac(Lam[1], -0.2892857142857143, Ops::mulc(Lam[0], -0.14464285714285716)))); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, -0.0060267857142857146, k); } y[5] = Ops::fma3(k, x[8], y[5]); y[8] = Ops::fma3(k, x[5], y[8]); }
    if constexpr (STIFF) { if constexpr (STIFF) { k = Ops::fmac(Lam[6], -0.2892857142857143, Ops::fmac(Lam[3], -0.14464285714285716, Ops::fmac(Lam[1], -0.14464285714285716, Ops::mulc(Lam[0], -0.14464285714285716)))); } else { k = Ops::zero(); } y[5] = Ops::fma3(k, x[9], y[5]); y[9] = Ops::fma3(k, x[5], y[9]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[5], 0.5785714285714286, Ops::fmac(Lam[4], 0.7232142857142857, Ops::fmac(Lam[2], 1.1571428571428573, Ops::mulc(Lam[1], 0.5785714285714286)))); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, 0.012053571428571429, k); } y[5] = Ops::fma3(k, x[10], y[5]); y[10] = Ops::fma3(k, x[5], y[10]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[5], -0.2892857142857143, Ops::fmac(Lam[4], -0.14464285714285716, Ops::fmac(Lam[2], -0.43392857142857144, Ops::mulc(Lam[1], -0.14464285714285716)))); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, -0.0060267857142857146, k); } y[5] = Ops::fma3(k, x[11], y[5]); y[11] = Ops::fma3(k, x[5], y[11]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[6], 0.5785714285714286, Ops::fmac(Lam[4], 0.7232142857142857, Ops::fmac(Lam[3], 1.1571428571428573, Ops::mulc(Lam[1], 0.5785714285714286)))); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, 0.012053571428571429, k); } y[5] = Ops::fma3(k, x[12], y[5]); y[12] = Ops::fma3(k, x[5], y[12]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[6], -0.2892857142857143, Ops::fmac(Lam[4], -0.14464285714285716, Ops::fmac(Lam[3], -0.43392857142857144, Ops::mulc(Lam[1], -0.14464285714285716)))); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, -0.0060267857142857146, k); } y[5] = Ops::fma3(k, x[13], y[5]); y[13] = Ops::fma3(k, x[5], y[13]); }
    if constexpr (STIFF) { if constexpr (STIFF) { k = Ops::fmac(Lam[6], -0.14464285714285716, Ops::fmac(Lam[5], -0.14464285714285716, Ops::fmac(Lam[3], -0.14464285714285716, Ops::mulc(Lam[2], -0.14464285714285716)))); } else { k = Ops::zero(); } y[5] = Ops::fma3(k, x[14], y[5]); y[14] = Ops::fma3(k, x[5], y[14]); }
    if constexpr (STIFF) { if constexpr (STIFF) { k = Ops::fmac(Lam[6], -0.14464285714285716, Ops::fmac(Lam[5], -0.14464285714285716, Ops::fmac(Lam[3], -0.14464285714285716, Ops::mulc(Lam[2], -0.14464285714285716)))); } else { k = Ops::zero(); } y[5] = Ops::fma3(k, x[15], y[5]); y[15] = Ops::fma3(k, x[5], y[15]); }
    if constexpr (STIFF) { if constexpr (STIFF) { k = Ops::fmac(Lam[5], 1.4464285714285714, Ops::fmac(Lam[4], -0.2892857142857143, Ops::fmac(Lam[2], 0.5785714285714286, Ops::fmac(Lam[1], 0.5785714285714286, Ops::mulc(Lam[0], 0.5785714285714286))))); } else { k = Ops::zero(); } y[5] = Ops::fma3(k, x[16], y[5]); y[16] = Ops::fma3(k, x[5], y[16]); }
    if constexpr (STIFF) { if constexpr (STIFF) { k = Ops::fmac(Lam[6], 1.4464285714285714, Ops::fmac(Lam[4], -0.2892857142857143, Ops::fmac(Lam[3], 0.5785714285714286, Ops::fmac(Lam[1], 0.5785714285714286, Ops::mulc(Lam[0], 0.5785714285714286))))); } else { k = Ops::zero(); } y[5] = Ops::fma3(k, x[17], y[5]); y[17] = Ops::fma3(k, x[5], y[17]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[6], -0.2892857142857143, Ops::fmac(Lam[5], -0.2892857142857143, Ops::fmac(Lam[3], -0.14464285714285716, Ops::fmac(Lam[2], -0.14464285714285716, Ops::fmac(Lam[1], -0.14464285714285716, Ops::mulc(Lam[0], -0.14464285714285716)))))); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, -0.012053571428571429, k); } y[5] = Ops::fma3(k, x[18], y[5]); y[18] = Ops::fma3(k, x[5], y[18]); }
    if constexpr (STIFF) { if constexpr (STIFF) { k = Ops::fmac(Lam[6], 0.7232142857142857, Ops::fmac(Lam[5], 0.7232142857142857, Ops::fmac(Lam[4], -0.14464285714285716, Ops::fmac(Lam[3], 0.5785714285714286, Ops::fmac(Lam[2], 0.5785714285714286, Ops::mulc(Lam[1], -0.14464285714285716)))))); } else { k = Ops::zero(); } y[5] = Ops::fma3(k, x[19], y[5]); y[19] = Ops::fma3(k, x[5], y[19]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[7], 1.1571428571428573, Ops::fmac(Lam[2], 1.1571428571428573, Ops::mulc(Lam[0], 1.4464285714285714))); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, 0.024107142857142858, k); } y[6] = Ops::fma3(k, x[6], y[6]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[7], -0.43392857142857144, Ops::fmac(Lam[2], 0.2892857142857143, Ops::mulc(Lam[0], -0.43392857142857144))); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, -0.012053571428571429, k); } y[6] = Ops::fma3(k, x[7], y[6]); y[7] = Ops::fma3(k, x[6], y[7]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[8], 1.1571428571428573, Ops::fmac(Lam[3], 0.5785714285714286, Ops::fmac(Lam[2], 0.5785714285714286, Ops::mulc(Lam[0], 0.7232142857142857)))); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, 0.012053571428571429, k); } y[6] = Ops::fma3(k, x[8], y[6]); y[8] = Ops::fma3(k, x[6], y[8]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[8], -0.43392857142857144, Ops::fmac(Lam[3], -0.2892857142857143, Ops::fmac(Lam[2], -0.14464285714285716, Ops::mulc(Lam[0], -0.14464285714285716)))); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, -0.0060267857142857146, k); } y[6] = Ops::fma3(k, x[9], y[6]); y[9] = Ops::fma3(k, x[6], y[9]); }
    if constexpr (STIFF) { if constexpr (STIFF) { k = Ops::fmac(Lam[7], -0.14464285714285716, Ops::fmac(Lam[5], -0.14464285714285716, Ops::fmac(Lam[2], -0.14464285714285716, Ops::mulc(Lam[1], -0.2892857142857143)))); } else { k = Ops::zero(); } y[6] = Ops::fma3(k, x[10], y[6]); y[10] = Ops::fma3(k, x[6], y[10]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[7], -0.14464285714285716, Ops::fmac(Lam[5], -0.14464285714285716, Ops::fmac(Lam[2], -0.2892857142857143, Ops::mulc(Lam[1], -0.43392857142857144)))); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, -0.0060267857142857146, k); } y[6] = Ops::fma3(k, x[11], y[6]); y[11] = Ops::fma3(k, x[6], y[11]); }
    if constexpr (STIFF) { if constexpr (STIFF) { k = Ops::fmac(Lam[8], -0.14464285714285716, Ops::fmac(Lam[5], -0.14464285714285716, Ops::fmac(Lam[3], -0.14464285714285716, Ops::mulc(Lam[1], -0.14464285714285716)))); } else { k = Ops::zero(); } y[6] = Ops::fma3(k, x[12], y[6]); y[12] = Ops::fma3(k, x[6], y[12]); }
    if constexpr (STIFF) { if constexpr (STIFF) { k = Ops::fmac(Lam[8], -0.14464285714285716, Ops::fmac(Lam[5], -0.14464285714285716, Ops::fmac(Lam[3], -0.14464285714285716, Ops::mulc(Lam[1], -0.14464285714285716)))); } else { k = Ops::zero(); } y[6] = Ops::fma3(k, x[13], y[6]); y[13] = Ops::fma3(k, x[6], y[13]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[8], -0.14464285714285716, Ops::fmac(Lam[7], -0.14464285714285716, Ops::fmac(Lam[3], -0.43392857142857144, Ops::mulc(Lam[2], -0.2892857142857143)))); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, -0.0060267857142857146, k); } y[6] = Ops::fma3(k, x[14], y[6]); y[14] = Ops::fma3(k, x[6], y[14]); }
    if constexpr (STIFF) { if constexpr (STIFF) { k = Ops::fmac(Lam[8], -0.14464285714285716, Ops::fmac(Lam[7], -0.14464285714285716, Ops::fmac(Lam[3], -0.2892857142857143, Ops::mulc(Lam[2], -0.14464285714285716)))); } else { k = Ops::zero(); } y[6] = Ops::fma3(k, x[15], y[6]); y[15] = Ops::fma3(k, x[6], y[15]); }
    if constexpr (STIFF) { if constexpr (STIFF) { k = Ops::fmac(Lam[7], 0.5785714285714286, Ops::fmac(Lam[5], 0.5785714285714286, Ops::fmac(Lam[2], 0.5785714285714286, Ops::fmac(Lam[1], 1.4464285714285714, Ops::mulc(Lam[0], -0.2892857142857143))))); } else { k = Ops::zero(); } y[6] = Ops::fma3(k, x[16], y[6]); y[16] = Ops::fma3(k, x[6], y[16]); }
    if constexpr (STIFF) { if constexpr (STIFF) { k = Ops::fmac(Lam[8], 0.5785714285714286, Ops::fmac(Lam[5], 0.5785714285714286, Ops::fmac(Lam[3], 0.7232142857142857, Ops::fmac(Lam[2], -0.14464285714285716, Ops::fmac(Lam[1], 0.7232142857142857, Ops::mulc(Lam[0], -0.14464285714285716)))))); } else { k = Ops::zero(); } y[6] = Ops::fma3(k, x[17], y[6]); y[17] = Ops::fma3(k, x[6], y[17]); }
    if constexpr (STIFF) { if constexpr (STIFF) { k = Ops::fmac(Lam[8], 0.5785714285714286, Ops::fmac(Lam[7], 0.5785714285714286, Ops::fmac(Lam[3], 1.4464285714285714, Ops::fmac(Lam[2], 0.5785714285714286, Ops::mulc(Lam[0], -0.2892857142857143))))); } else { k = Ops::zero(); } y[6] = Ops::fma3(k, x[18], y[6]); y[18] = Ops::fma3(k, x[6], y[18]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[8], -0.14464285714285716, Ops::fmac(Lam[7], -0.14464285714285716, Ops::fmac(Lam[5], -0.14464285714285716, Ops::fmac(Lam[3], -0.2892857142857143, Ops::fmac(Lam[2], -0.14464285714285716, Ops::mulc(Lam[1], -0.2892857142857143)))))); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, -0.012053571428571429, k); } y[6] = Ops::fma3(k, x[19], y[6]); y[19] = Ops::fma3(k, x[6], y[19]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[7], 1.4464285714285714, Ops::fmac(Lam[2], 1.1571428571428573, Ops::mulc(Lam[0], 1.1571428571428573))); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, 0.024107142857142858, k); } y[7] = Ops::fma3(k, x[7], y[7]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[8], -0.43392857142857144, Ops::fmac(Lam[3], -0.14464285714285716, Ops::fmac(Lam[2], -0.2892857142857143, Ops::mulc(Lam[0], -0.14464285714285716)))); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, -0.0060267857142857146, k); } y[7] = Ops::fma3(k, x[8], y[7]); y[8] = Ops::fma3(k, x[7], y[8]); }
    if constexpr (STIFF) { if constexpr (STIFF) { k = Ops::fmac(Lam[8], -0.2892857142857143, Ops::fmac(Lam[3], -0.14464285714285716, Ops::fmac(Lam[2], -0.14464285714285716, Ops::mulc(Lam[0], -0.14464285714285716)))); } else { k = Ops::zero(); } y[7] = Ops::fma3(k, x[9], y[7]); y[9] = Ops::fma3(k, x[7], y[9]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[7], -0.14464285714285716, Ops::fmac(Lam[5], -0.2892857142857143, Ops::fmac(Lam[2], -0.14464285714285716, Ops::mulc(Lam[1], -0.43392857142857144)))); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, -0.0060267857142857146, k); } y[7] = Ops::fma3(k, x[10], y[7]); y[10] = Ops::fma3(k, x[7], y[10]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[7], 0.7232142857142857, Ops::fmac(Lam[5], 0.5785714285714286, Ops::fmac(Lam[2], 0.5785714285714286, Ops::mulc(Lam[1], 1.1571428571428573)))); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, 0.012053571428571429, k); } y[7] = Ops::fma3(k, x[11], y[7]); y[11] = Ops::fma3(k, x[7], y[11]); }
    if constexpr (STIFF) { if constexpr (STIFF) { k = Ops::fmac(Lam[8], -0.14464285714285716, Ops::fmac(Lam[5], -0.14464285714285716, Ops::fmac(Lam[3], -0.14464285714285716, Ops::mulc(Lam[1], -0.14464285714285716)))); } else { k = Ops::zero(); } y[7] = Ops::fma3(k, x[12], y[7]); y[12] = Ops::fma3(k, x[7], y[12]); }
    if constexpr (STIFF) { if constexpr (STIFF) { k = Ops::fmac(Lam[8], -0.14464285714285716, Ops::fmac(Lam[5], -0.14464285714285716, Ops::fmac(Lam[3], -0.14464285714285716, Ops::mulc(Lam[1], -0.14464285714285716)))); } else { k = Ops::zero(); } y[7] = Ops::fma3(k, x[13], y[7]); y[13] = Ops::fma3(k, x[7], y[13]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[8], 0.5785714285714286, Ops::fmac(Lam[7], 0.7232142857142857, Ops::fmac(Lam[3], 1.1571428571428573, Ops::mulc(Lam[2], 0.5785714285714286)))); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, 0.012053571428571429, k); } y[7] = Ops::fma3(k, x[14], y[7]); y[14] = Ops::fma3(k, x[7], y[14]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[8], -0.2892857142857143, Ops::fmac(Lam[7], -0.14464285714285716, Ops::fmac(Lam[3], -0.43392857142857144, Ops::mulc(Lam[2], -0.14464285714285716)))); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, -0.0060267857142857146, k); } y[7] = Ops::fma3(k, x[15], y[7]); y[15] = Ops::fma3(k, x[7], y[15]); }
    if constexpr (STIFF) { if constexpr (STIFF) { k = Ops::fmac(Lam[7], -0.2892857142857143, Ops::fmac(Lam[5], 1.4464285714285714, Ops::fmac(Lam[2], 0.5785714285714286, Ops::fmac(Lam[1], 0.5785714285714286, Ops::mulc(Lam[0], 0.5785714285714286))))); } else { k = Ops::zero(); } y[7] = Ops::fma3(k, x[16], y[7]); y[16] = Ops::fma3(k, x[7], y[16]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[8], -0.2892857142857143, Ops::fmac(Lam[5], -0.2892857142857143, Ops::fmac(Lam[3], -0.14464285714285716, Ops::fmac(Lam[2], -0.14464285714285716, Ops::fmac(Lam[1], -0.14464285714285716, Ops::mulc(Lam[0], -0.14464285714285716)))))); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, -0.012053571428571429, k); } y[7] = Ops::fma3(k, x[17], y[7]); y[17] = Ops::fma3(k, x[7], y[17]); }
    if constexpr (STIFF) { if constexpr (STIFF) { k = Ops::fmac(Lam[8], 1.4464285714285714, Ops::fmac(Lam[7], -0.2892857142857143, Ops::fmac(Lam[3], 0.5785714285714286, Ops::fmac(Lam[2], 0.5785714285714286, Ops::mulc(Lam[0], 0.5785714285714286))))); } else { k = Ops::zero(); } y[7] = Ops::fma3(k, x[18], y[7]); y[18] = Ops::fma3(k, x[7], y[18]); }
    if constexpr (STIFF) { if constexpr (STIFF) { k = Ops::fmac(Lam[8], 0.7232142857142857, Ops::fmac(Lam[7], -0.14464285714285716, Ops::fmac(Lam[5], 0.7232142857142857, Ops::fmac(Lam[3], 0.5785714285714286, Ops::fmac(Lam[2], -0.14464285714285716, Ops::mulc(Lam[1], 0.5785714285714286)))))); } else { k = Ops::zero(); } y[7] = Ops::fma3(k, x[19], y[7]); y[19] = Ops::fma3(k, x[7], y[19]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[9], 1.1571428571428573, Ops::fmac(Lam[3], 1.1571428571428573, Ops::mulc(Lam[0], 1.4464285714285714))); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, 0.024107142857142858, k); } y[8] = Ops::fma3(k, x[8], y[8]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[9], -0.43392857142857144, Ops::fmac(Lam[3], 0.2892857142857143, Ops::mulc(Lam[0], -0.43392857142857144))); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, -0.012053571428571429, k); } y[8] = Ops::fma3(k, x[9], y[8]); y[9] = Ops::fma3(k, x[8], y[9]); }
    if constexpr (STIFF) { if constexpr (STIFF) { k = Ops::fmac(Lam[8], -0.14464285714285716, Ops::fmac(Lam[6], -0.14464285714285716, Ops::fmac(Lam[2], -0.14464285714285716, Ops::mulc(Lam[1], -0.14464285714285716)))); } else { k = Ops::zero(); } y[8] = Ops::fma3(k, x[10], y[8]); y[10] = Ops::fma3(k, x[8], y[10]); }
    if constexpr (STIFF) { if constexpr (STIFF) { k = Ops::fmac(Lam[8], -0.14464285714285716, Ops::fmac(Lam[6], -0.14464285714285716, Ops::fmac(Lam[2], -0.14464285714285716, Ops::mulc(Lam[1], -0.14464285714285716)))); } else { k = Ops::zero(); } y[8] = Ops::fma3(k, x[11], y[8]); y[11] = Ops::fma3(k, x[8], y[11]); }
    if constexpr (STIFF) { if constexpr (STIFF) { k = Ops::fmac(Lam[9], -0.14464285714285716, Ops::fmac(Lam[6], -0.14464285714285716, Ops::fmac(Lam[3], -0.14464285714285716, Ops::mulc(Lam[1], -0.2892857142857143)))); } else { k = Ops::zero(); } y[8] = Ops::fma3(k, x[12], y[8]); y[12] = Ops::fma3(k, x[8], y[12]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[9], -0.14464285714285716, Ops::fmac(Lam[6], -0.14464285714285716, Ops::fmac(Lam[3], -0.2892857142857143, Ops::mulc(Lam[1], -0.43392857142857144)))); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, -0.0060267857142857146, k); } y[8] = Ops::fma3(k, x[13], y[8]); y[13] = Ops::fma3(k, x[8], y[13]); }
    if constexpr (STIFF) { if constexpr (STIFF) { k = Ops::fmac(Lam[9], -0.14464285714285716, Ops::fmac(Lam[8], -0.14464285714285716, Ops::fmac(Lam[3], -0.14464285714285716, Ops::mulc(Lam[2], -0.2892857142857143)))); } else { k = Ops::zero(); } y[8] = Ops::fma3(k, x[14], y[8]); y[14] = Ops::fma3(k, x[8], y[14]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[9], -0.14464285714285716, Ops::fmac(Lam[8], -0.14464285714285716, Ops::fmac(Lam[3], -0.2892857142857143, Ops::mulc(Lam[2], -0.43392857142857144)))); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, -0.0060267857142857146, k); } y[8] = Ops::fma3(k, x[15], y[8]); y[15] = Ops::fma3(k, x[8], y[15]); }
    if constexpr (STIFF) { if constexpr (STIFF) { k = Ops::fmac(Lam[8], 0.5785714285714286, Ops::fmac(Lam[6], 0.5785714285714286, Ops::fmac(Lam[3], -0.14464285714285716, Ops::fmac(Lam[2], 0.7232142857142857, Ops::fmac(Lam[1], 0.7232142857142857, Ops::mulc(Lam[0], -0.14464285714285716)))))); } else { k = Ops::zero(); } y[8] = Ops::fma3(k, x[16], y[8]); y[16] = Ops::fma3(k, x[8], y[16]); }
    if constexpr (STIFF) { if constexpr (STIFF) { k = Ops::fmac(Lam[9], 0.5785714285714286, Ops::fmac(Lam[6], 0.5785714285714286, Ops::fmac(Lam[3], 0.5785714285714286, Ops::fmac(Lam[1], 1.4464285714285714, Ops::mulc(Lam[0], -0.2892857142857143))))); } else { k = Ops::zero(); } y[8] = Ops::fma3(k, x[17], y[8]); y[17] = Ops::fma3(k, x[8], y[17]); }
    if constexpr (STIFF) { if constexpr (STIFF) { k = Ops::fmac(Lam[9], 0.5785714285714286, Ops::fmac(Lam[8], 0.5785714285714286, Ops::fmac(Lam[3], 0.5785714285714286, Ops::fmac(Lam[2], 1.4464285714285714, Ops::mulc(Lam[0], -0.2892857142857143))))); } else { k = Ops::zero(); } y[8] = Ops::fma3(k, x[18], y[8]); y[18] = Ops::fma3(k, x[8], y[18]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[9], -0.14464285714285716, Ops::fmac(Lam[8], -0.14464285714285716, Ops::fmac(Lam[6], -0.14464285714285716, Ops::fmac(Lam[3], -0.14464285714285716, Ops::fmac(Lam[2], -0.2892857142857143, Ops::mulc(Lam[1], -0.2892857142857143)))))); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, -0.012053571428571429, k); } y[8] = Ops::fma3(k, x[19], y[8]); y[19] = Ops::fma3(k, x[8], y[19]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[9], 1.4464285714285714, Ops::fmac(Lam[3], 1.1571428571428573, Ops::mulc(Lam[0], 1.1571428571428573))); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, 0.024107142857142858, k); } y[9] = Ops::fma3(k, x[9], y[9]); }
    if constexpr (STIFF) { if constexpr (STIFF) { k = Ops::fmac(Lam[8], -0.14464285714285716, Ops::fmac(Lam[6], -0.14464285714285716, Ops::fmac(Lam[2], -0.14464285714285716, Ops::mulc(Lam[1], -0.14464285714285716)))); } else { k = Ops::zero(); } y[9] = Ops::fma3(k, x[10], y[9]); y[10] = Ops::fma3(k, x[9], y[10]); }
    if constexpr (STIFF) { if constexpr (STIFF) { k = Ops::fmac(Lam[8], -0.14464285714285716, Ops::fmac(Lam[6], -0.14464285714285716, Ops::fmac(Lam[2], -0.14464285714285716, Ops::mulc(Lam[1], -0.14464285714285716)))); } else { k = Ops::zero(); } y[9] = Ops::fma3(k, x[11], y[9]); y[11] = Ops::fma3(k, x[9], y[11]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[9], -0.14464285714285716, Ops::fmac(Lam[6], -0.2892857142857143, Ops::fmac(Lam[3], -0.14464285714285716, Ops::mulc(Lam[1], -0.43392857142857144)))); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, -0.0060267857142857146, k); } y[9] = Ops::fma3(k, x[12], y[9]); y[12] = Ops::fma3(k, x[9], y[12]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[9], 0.7232142857142857, Ops::fmac(Lam[6], 0.5785714285714286, Ops::fmac(Lam[3], 0.5785714285714286, Ops::mulc(Lam[1], 1.1571428571428573)))); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, 0.012053571428571429, k); } y[9] = Ops::fma3(k, x[13], y[9]); y[13] = Ops::fma3(k, x[9], y[13]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[9], -0.14464285714285716, Ops::fmac(Lam[8], -0.2892857142857143, Ops::fmac(Lam[3], -0.14464285714285716, Ops::mulc(Lam[2], -0.43392857142857144)))); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, -0.0060267857142857146, k); } y[9] = Ops::fma3(k, x[14], y[9]); y[14] = Ops::fma3(k, x[9], y[14]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[9], 0.7232142857142857, Ops::fmac(Lam[8], 0.5785714285714286, Ops::fmac(Lam[3], 0.5785714285714286, Ops::mulc(Lam[2], 1.1571428571428573)))); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, 0.012053571428571429, k); } y[9] = Ops::fma3(k, x[15], y[9]); y[15] = Ops::fma3(k, x[9], y[15]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[8], -0.2892857142857143, Ops::fmac(Lam[6], -0.2892857142857143, Ops::fmac(Lam[3], -0.14464285714285716, Ops::fmac(Lam[2], -0.14464285714285716, Ops::fmac(Lam[1], -0.14464285714285716, Ops::mulc(Lam[0], -0.14464285714285716)))))); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, -0.012053571428571429, k); } y[9] = Ops::fma3(k, x[16], y[9]); y[16] = Ops::fma3(k, x[9], y[16]); }
    if constexpr (STIFF) { if constexpr (STIFF) { k = Ops::fmac(Lam[9], -0.2892857142857143, Ops::fmac(Lam[6], 1.4464285714285714, Ops::fmac(Lam[3], 0.5785714285714286, Ops::fmac(Lam[1], 0.5785714285714286, Ops::mulc(Lam[0], 0.5785714285714286))))); } else { k = Ops::zero(); } y[9] = Ops::fma3(k, x[17], y[9]); y[17] = Ops::fma3(k, x[9], y[17]); }
    if constexpr (STIFF) { if constexpr (STIFF) { k = Ops::fmac(Lam[9], -0.2892857142857143, Ops::fmac(Lam[8], 1.4464285714285714, Ops::fmac(Lam[3], 0.5785714285714286, Ops::fmac(Lam[2], 0.5785714285714286, Ops::mulc(Lam[0], 0.5785714285714286))))); } else { k = Ops::zero(); } y[9] = Ops::fma3(k, x[18], y[9]); y[18] = Ops::fma3(k, x[9], y[18]); }
    if constexpr (STIFF) { if constexpr (STIFF) { k = Ops::fmac(Lam[9], -0.14464285714285716, Ops::fmac(Lam[8], 0.7232142857142857, Ops::fmac(Lam[6], 0.7232142857142857, Ops::fmac(Lam[3], -0.14464285714285716, Ops::fmac(Lam[2], 0.5785714285714286, Ops::mulc(Lam[1], 0.5785714285714286)))))); } else { k = Ops::zero(); } y[9] = Ops::fma3(k, x[19], y[9]); y[19] = Ops::fma3(k, x[9], y[19]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[7], 1.1571428571428573, Ops::fmac(Lam[5], 1.1571428571428573, Ops::mulc(Lam[4], 1.4464285714285714))); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, 0.024107142857142858, k); } y[10] = Ops::fma3(k, x[10], y[10]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[7], -0.43392857142857144, Ops::fmac(Lam[5], 0.2892857142857143, Ops::mulc(Lam[4], -0.43392857142857144))); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, -0.012053571428571429, k); } y[10] = Ops::fma3(k, x[11], y[10]); y[11] = Ops::fma3(k, x[10], y[11]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[8], 1.1571428571428573, Ops::fmac(Lam[6], 0.5785714285714286, Ops::fmac(Lam[5], 0.5785714285714286, Ops::mulc(Lam[4], 0.7232142857142857)))); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, 0.012053571428571429, k); } y[10] = Ops::fma3(k, x[12], y[10]); y[12] = Ops::fma3(k, x[10], y[12]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[8], -0.43392857142857144, Ops::fmac(Lam[6], -0.2892857142857143, Ops::fmac(Lam[5], -0.14464285714285716, Ops::mulc(Lam[4], -0.14464285714285716)))); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, -0.0060267857142857146, k); } y[10] = Ops::fma3(k, x[13], y[10]); y[13] = Ops::fma3(k, x[10], y[13]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[8], -0.14464285714285716, Ops::fmac(Lam[7], -0.14464285714285716, Ops::fmac(Lam[6], -0.43392857142857144, Ops::mulc(Lam[5], -0.2892857142857143)))); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, -0.0060267857142857146, k); } y[10] = Ops::fma3(k, x[14], y[10]); y[14] = Ops::fma3(k, x[10], y[14]); }
    if constexpr (STIFF) { if constexpr (STIFF) { k = Ops::fmac(Lam[8], -0.14464285714285716, Ops::fmac(Lam[7], -0.14464285714285716, Ops::fmac(Lam[6], -0.2892857142857143, Ops::mulc(Lam[5], -0.14464285714285716)))); } else { k = Ops::zero(); } y[10] = Ops::fma3(k, x[15], y[10]); y[15] = Ops::fma3(k, x[10], y[15]); }
    if constexpr (STIFF) { if constexpr (STIFF) { k = Ops::fmac(Lam[7], 0.5785714285714286, Ops::fmac(Lam[5], 0.5785714285714286, Ops::fmac(Lam[4], -0.2892857142857143, Ops::fmac(Lam[2], 0.5785714285714286, Ops::mulc(Lam[1], 1.4464285714285714))))); } else { k = Ops::zero(); } y[10] = Ops::fma3(k, x[16], y[10]); y[16] = Ops::fma3(k, x[10], y[16]); }
    if constexpr (STIFF) { if constexpr (STIFF) { k = Ops::fmac(Lam[8], 0.5785714285714286, Ops::fmac(Lam[6], 0.7232142857142857, Ops::fmac(Lam[5], -0.14464285714285716, Ops::fmac(Lam[4], -0.14464285714285716, Ops::fmac(Lam[2], 0.5785714285714286, Ops::mulc(Lam[1], 0.7232142857142857)))))); } else { k = Ops::zero(); } y[10] = Ops::fma3(k, x[17], y[10]); y[17] = Ops::fma3(k, x[10], y[17]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[8], -0.14464285714285716, Ops::fmac(Lam[7], -0.14464285714285716, Ops::fmac(Lam[6], -0.2892857142857143, Ops::fmac(Lam[5], -0.14464285714285716, Ops::fmac(Lam[2], -0.14464285714285716, Ops::mulc(Lam[1], -0.2892857142857143)))))); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, -0.012053571428571429, k); } y[10] = Ops::fma3(k, x[18], y[10]); y[18] = Ops::fma3(k, x[10], y[18]); }
    if constexpr (STIFF) { if constexpr (STIFF) { k = Ops::fmac(Lam[8], 0.5785714285714286, Ops::fmac(Lam[7], 0.5785714285714286, Ops::fmac(Lam[6], 1.4464285714285714, Ops::fmac(Lam[5], 0.5785714285714286, Ops::mulc(Lam[4], -0.2892857142857143))))); } else { k = Ops::zero(); } y[10] = Ops::fma3(k, x[19], y[10]); y[19] = Ops::fma3(k, x[10], y[19]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[7], 1.4464285714285714, Ops::fmac(Lam[5], 1.1571428571428573, Ops::mulc(Lam[4], 1.1571428571428573))); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, 0.024107142857142858, k); } y[11] = Ops::fma3(k, x[11], y[11]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[8], -0.43392857142857144, Ops::fmac(Lam[6], -0.14464285714285716, Ops::fmac(Lam[5], -0.2892857142857143, Ops::mulc(Lam[4], -0.14464285714285716)))); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, -0.0060267857142857146, k); } y[11] = Ops::fma3(k, x[12], y[11]); y[12] = Ops::fma3(k, x[11], y[12]); }
    if constexpr (STIFF) { if constexpr (STIFF) { k = Ops::fmac(Lam[8], -0.2892857142857143, Ops::fmac(Lam[6], -0.14464285714285716, Ops::fmac(Lam[5], -0.14464285714285716, Ops::mulc(Lam[4], -0.14464285714285716)))); } else { k = Ops::zero(); } y[11] = Ops::fma3(k, x[13], y[11]); y[13] = Ops::fma3(k, x[11], y[13]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[8], 0.5785714285714286, Ops::fmac(Lam[7], 0.7232142857142857, Ops::fmac(Lam[6], 1.1571428571428573, Ops::mulc(Lam[5], 0.5785714285714286)))); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, 0.012053571428571429, k); } y[11] = Ops::fma3(k, x[14], y[11]); y[14] = Ops::fma3(k, x[11], y[14]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[8], -0.2892857142857143, Ops::fmac(Lam[7], -0.14464285714285716, Ops::fmac(Lam[6], -0.43392857142857144, Ops::mulc(Lam[5], -0.14464285714285716)))); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, -0.0060267857142857146, k); } y[11] = Ops::fma3(k, x[15], y[11]); y[15] = Ops::fma3(k, x[11], y[15]); }
    if constexpr (STIFF) { if constexpr (STIFF) { k = Ops::fmac(Lam[7], -0.2892857142857143, Ops::fmac(Lam[5], 0.5785714285714286, Ops::fmac(Lam[4], 0.5785714285714286, Ops::fmac(Lam[2], 1.4464285714285714, Ops::mulc(Lam[1], 0.5785714285714286))))); } else { k = Ops::zero(); } y[11] = Ops::fma3(k, x[16], y[11]); y[16] = Ops::fma3(k, x[11], y[16]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[8], -0.2892857142857143, Ops::fmac(Lam[6], -0.14464285714285716, Ops::fmac(Lam[5], -0.14464285714285716, Ops::fmac(Lam[4], -0.14464285714285716, Ops::fmac(Lam[2], -0.2892857142857143, Ops::mulc(Lam[1], -0.14464285714285716)))))); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, -0.012053571428571429, k); } y[11] = Ops::fma3(k, x[17], y[11]); y[17] = Ops::fma3(k, x[11], y[17]); }
    if constexpr (STIFF) { if constexpr (STIFF) { k = Ops::fmac(Lam[8], 0.7232142857142857, Ops::fmac(Lam[7], -0.14464285714285716, Ops::fmac(Lam[6], 0.5785714285714286, Ops::fmac(Lam[5], -0.14464285714285716, Ops::fmac(Lam[2], 0.7232142857142857, Ops::mulc(Lam[1], 0.5785714285714286)))))); } else { k = Ops::zero(); } y[11] = Ops::fma3(k, x[18], y[11]); y[18] = Ops::fma3(k, x[11], y[18]); }
    if constexpr (STIFF) { if constexpr (STIFF) { k = Ops::fmac(Lam[8], 1.4464285714285714, Ops::fmac(Lam[7], -0.2892857142857143, Ops::fmac(Lam[6], 0.5785714285714286, Ops::fmac(Lam[5], 0.5785714285714286, Ops::mulc(Lam[4], 0.5785714285714286))))); } else { k = Ops::zero(); } y[11] = Ops::fma3(k, x[19], y[11]); y[19] = Ops::fma3(k, x[11], y[19]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[9], 1.1571428571428573, Ops::fmac(Lam[6], 1.1571428571428573, Ops::mulc(Lam[4], 1.4464285714285714))); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, 0.024107142857142858, k); } y[12] = Ops::fma3(k, x[12], y[12]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[9], -0.43392857142857144, Ops::fmac(Lam[6], 0.2892857142857143, Ops::mulc(Lam[4], -0.43392857142857144))); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, -0.012053571428571429, k); } y[12] = Ops::fma3(k, x[13], y[12]); y[13] = Ops::fma3(k, x[12], y[13]); }
    if constexpr (STIFF) { if constexpr (STIFF) { k = Ops::fmac(Lam[9], -0.14464285714285716, Ops::fmac(Lam[8], -0.14464285714285716, Ops::fmac(Lam[6], -0.14464285714285716, Ops::mulc(Lam[5], -0.2892857142857143)))); } else { k = Ops::zero(); } y[12] = Ops::fma3(k, x[14], y[12]); y[14] = Ops::fma3(k, x[12], y[14]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[9], -0.14464285714285716, Ops::fmac(Lam[8], -0.14464285714285716, Ops::fmac(Lam[6], -0.2892857142857143, Ops::mulc(Lam[5], -0.43392857142857144)))); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, -0.0060267857142857146, k); } y[12] = Ops::fma3(k, x[15], y[12]); y[15] = Ops::fma3(k, x[12], y[15]); }
    if constexpr (STIFF) { if constexpr (STIFF) { k = Ops::fmac(Lam[8], 0.5785714285714286, Ops::fmac(Lam[6], -0.14464285714285716, Ops::fmac(Lam[5], 0.7232142857142857, Ops::fmac(Lam[4], -0.14464285714285716, Ops::fmac(Lam[3], 0.5785714285714286, Ops::mulc(Lam[1], 0.7232142857142857)))))); } else { k = Ops::zero(); } y[12] = Ops::fma3(k, x[16], y[12]); y[16] = Ops::fma3(k, x[12], y[16]); }
    if constexpr (STIFF) { if constexpr (STIFF) { k = Ops::fmac(Lam[9], 0.5785714285714286, Ops::fmac(Lam[6], 0.5785714285714286, Ops::fmac(Lam[4], -0.2892857142857143, Ops::fmac(Lam[3], 0.5785714285714286, Ops::mulc(Lam[1], 1.4464285714285714))))); } else { k = Ops::zero(); } y[12] = Ops::fma3(k, x[17], y[12]); y[17] = Ops::fma3(k, x[12], y[17]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[9], -0.14464285714285716, Ops::fmac(Lam[8], -0.14464285714285716, Ops::fmac(Lam[6], -0.14464285714285716, Ops::fmac(Lam[5], -0.2892857142857143, Ops::fmac(Lam[3], -0.14464285714285716, Ops::mulc(Lam[1], -0.2892857142857143)))))); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, -0.012053571428571429, k); } y[12] = Ops::fma3(k, x[18], y[12]); y[18] = Ops::fma3(k, x[12], y[18]); }
    if constexpr (STIFF) { if constexpr (STIFF) { k = Ops::fmac(Lam[9], 0.5785714285714286, Ops::fmac(Lam[8], 0.5785714285714286, Ops::fmac(Lam[6], 0.5785714285714286, Ops::fmac(Lam[5], 1.4464285714285714, Ops::mulc(Lam[4], -0.2892857142857143))))); } else { k = Ops::zero(); } y[12] = Ops::fma3(k, x[19], y[12]); y[19] = Ops::fma3(k, x[12], y[19]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[9], 1.4464285714285714, Ops::fmac(Lam[6], 1.1571428571428573, Ops::mulc(Lam[4], 1.1571428571428573))); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, 0.024107142857142858, k); } y[13] = Ops::fma3(k, x[13], y[13]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[9], -0.14464285714285716, Ops::fmac(Lam[8], -0.2892857142857143, Ops::fmac(Lam[6], -0.14464285714285716, Ops::mulc(Lam[5], -0.43392857142857144)))); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, -0.0060267857142857146, k); } y[13] = Ops::fma3(k, x[14], y[13]); y[14] = Ops::fma3(k, x[13], y[14]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[9], 0.7232142857142857, Ops::fmac(Lam[8], 0.5785714285714286, Ops::fmac(Lam[6], 0.5785714285714286, Ops::mulc(Lam[5], 1.1571428571428573)))); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, 0.012053571428571429, k); } y[13] = Ops::fma3(k, x[15], y[13]); y[15] = Ops::fma3(k, x[13], y[15]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[8], -0.2892857142857143, Ops::fmac(Lam[6], -0.14464285714285716, Ops::fmac(Lam[5], -0.14464285714285716, Ops::fmac(Lam[4], -0.14464285714285716, Ops::fmac(Lam[3], -0.2892857142857143, Ops::mulc(Lam[1], -0.14464285714285716)))))); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, -0.012053571428571429, k); } y[13] = Ops::fma3(k, x[16], y[13]); y[16] = Ops::fma3(k, x[13], y[16]); }
    if constexpr (STIFF) { if constexpr (STIFF) { k = Ops::fmac(Lam[9], -0.2892857142857143, Ops::fmac(Lam[6], 0.5785714285714286, Ops::fmac(Lam[4], 0.5785714285714286, Ops::fmac(Lam[3], 1.4464285714285714, Ops::mulc(Lam[1], 0.5785714285714286))))); } else { k = Ops::zero(); } y[13] = Ops::fma3(k, x[17], y[13]); y[17] = Ops::fma3(k, x[13], y[17]); }
    if constexpr (STIFF) { if constexpr (STIFF) { k = Ops::fmac(Lam[9], -0.14464285714285716, Ops::fmac(Lam[8], 0.7232142857142857, Ops::fmac(Lam[6], -0.14464285714285716, Ops::fmac(Lam[5], 0.5785714285714286, Ops::fmac(Lam[3], 0.7232142857142857, Ops::mulc(Lam[1], 0.5785714285714286)))))); } else { k = Ops::zero(); } y[13] = Ops::fma3(k, x[18], y[13]); y[18] = Ops::fma3(k, x[13], y[18]); }
    if constexpr (STIFF) { if constexpr (STIFF) { k = Ops::fmac(Lam[9], -0.2892857142857143, Ops::fmac(Lam[8], 1.4464285714285714, Ops::fmac(Lam[6], 0.5785714285714286, Ops::fmac(Lam[5], 0.5785714285714286, Ops::mulc(Lam[4], 0.5785714285714286))))); } else { k = Ops::zero(); } y[13] = Ops::fma3(k, x[19], y[13]); y[19] = Ops::fma3(k, x[13], y[19]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[9], 1.1571428571428573, Ops::fmac(Lam[8], 1.1571428571428573, Ops::mulc(Lam[7], 1.4464285714285714))); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, 0.024107142857142858, k); } y[14] = Ops::fma3(k, x[14], y[14]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[9], -0.43392857142857144, Ops::fmac(Lam[8], 0.2892857142857143, Ops::mulc(Lam[7], -0.43392857142857144))); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, -0.012053571428571429, k); } y[14] = Ops::fma3(k, x[15], y[14]); y[15] = Ops::fma3(k, x[14], y[15]); }
    if constexpr (STIFF) { if constexpr (STIFF) { k = Ops::fmac(Lam[8], -0.14464285714285716, Ops::fmac(Lam[7], -0.14464285714285716, Ops::fmac(Lam[6], 0.5785714285714286, Ops::fmac(Lam[5], 0.7232142857142857, Ops::fmac(Lam[3], 0.5785714285714286, Ops::mulc(Lam[2], 0.7232142857142857)))))); } else { k = Ops::zero(); } y[14] = Ops::fma3(k, x[16], y[14]); y[16] = Ops::fma3(k, x[14], y[16]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[9], -0.14464285714285716, Ops::fmac(Lam[8], -0.14464285714285716, Ops::fmac(Lam[6], -0.14464285714285716, Ops::fmac(Lam[5], -0.2892857142857143, Ops::fmac(Lam[3], -0.14464285714285716, Ops::mulc(Lam[2], -0.2892857142857143)))))); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, -0.012053571428571429, k); } y[14] = Ops::fma3(k, x[17], y[14]); y[17] = Ops::fma3(k, x[14], y[17]); }
    if constexpr (STIFF) { if constexpr (STIFF) { k = Ops::fmac(Lam[9], 0.5785714285714286, Ops::fmac(Lam[8], 0.5785714285714286, Ops::fmac(Lam[7], -0.2892857142857143, Ops::fmac(Lam[3], 0.5785714285714286, Ops::mulc(Lam[2], 1.4464285714285714))))); } else { k = Ops::zero(); } y[14] = Ops::fma3(k, x[18], y[14]); y[18] = Ops::fma3(k, x[14], y[18]); }
    if constexpr (STIFF) { if constexpr (STIFF) { k = Ops::fmac(Lam[9], 0.5785714285714286, Ops::fmac(Lam[8], 0.5785714285714286, Ops::fmac(Lam[7], -0.2892857142857143, Ops::fmac(Lam[6], 0.5785714285714286, Ops::mulc(Lam[5], 1.4464285714285714))))); } else { k = Ops::zero(); } y[14] = Ops::fma3(k, x[19], y[14]); y[19] = Ops::fma3(k, x[14], y[19]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[9], 1.4464285714285714, Ops::fmac(Lam[8], 1.1571428571428573, Ops::mulc(Lam[7], 1.1571428571428573))); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, 0.024107142857142858, k); } y[15] = Ops::fma3(k, x[15], y[15]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[8], -0.14464285714285716, Ops::fmac(Lam[7], -0.14464285714285716, Ops::fmac(Lam[6], -0.2892857142857143, Ops::fmac(Lam[5], -0.14464285714285716, Ops::fmac(Lam[3], -0.2892857142857143, Ops::mulc(Lam[2], -0.14464285714285716)))))); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, -0.012053571428571429, k); } y[15] = Ops::fma3(k, x[16], y[15]); y[16] = Ops::fma3(k, x[15], y[16]); }
    if constexpr (STIFF) { if constexpr (STIFF) { k = Ops::fmac(Lam[9], -0.14464285714285716, Ops::fmac(Lam[8], -0.14464285714285716, Ops::fmac(Lam[6], 0.7232142857142857, Ops::fmac(Lam[5], 0.5785714285714286, Ops::fmac(Lam[3], 0.7232142857142857, Ops::mulc(Lam[2], 0.5785714285714286)))))); } else { k = Ops::zero(); } y[15] = Ops::fma3(k, x[17], y[15]); y[17] = Ops::fma3(k, x[15], y[17]); }
    if constexpr (STIFF) { if constexpr (STIFF) { k = Ops::fmac(Lam[9], -0.2892857142857143, Ops::fmac(Lam[8], 0.5785714285714286, Ops::fmac(Lam[7], 0.5785714285714286, Ops::fmac(Lam[3], 1.4464285714285714, Ops::mulc(Lam[2], 0.5785714285714286))))); } else { k = Ops::zero(); } y[15] = Ops::fma3(k, x[18], y[15]); y[18] = Ops::fma3(k, x[15], y[18]); }
    if constexpr (STIFF) { if constexpr (STIFF) { k = Ops::fmac(Lam[9], -0.2892857142857143, Ops::fmac(Lam[8], 0.5785714285714286, Ops::fmac(Lam[7], 0.5785714285714286, Ops::fmac(Lam[6], 1.4464285714285714, Ops::mulc(Lam[5], 0.5785714285714286))))); } else { k = Ops::zero(); } y[15] = Ops::fma3(k, x[19], y[15]); y[19] = Ops::fma3(k, x[15], y[19]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[7], 3.4714285714285715, Ops::fmac(Lam[5], 3.4714285714285715, Ops::fmac(Lam[4], 3.4714285714285715, Ops::fmac(Lam[2], 3.4714285714285715, Ops::fmac(Lam[1], 3.4714285714285715, Ops::mulc(Lam[0], 3.4714285714285715)))))); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, 0.09642857142857143, k); } y[16] = Ops::fma3(k, x[16], y[16]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[8], 3.4714285714285715, Ops::fmac(Lam[6], 1.7357142857142858, Ops::fmac(Lam[5], 1.7357142857142858, Ops::fmac(Lam[4], 1.7357142857142858, Ops::fmac(Lam[3], 1.7357142857142858, Ops::fmac(Lam[2], 1.7357142857142858, Ops::fmac(Lam[1], 1.7357142857142858, Ops::mulc(Lam[0], 1.7357142857142858)))))))); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, 0.048214285714285716, k); } y[16] = Ops::fma3(k, x[17], y[16]); y[17] = Ops::fma3(k, x[16], y[17]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[8], 1.7357142857142858, Ops::fmac(Lam[7], 1.7357142857142858, Ops::fmac(Lam[6], 3.4714285714285715, Ops::fmac(Lam[5], 1.7357142857142858, Ops::fmac(Lam[3], 1.7357142857142858, Ops::fmac(Lam[2], 1.7357142857142858, Ops::fmac(Lam[1], 1.7357142857142858, Ops::mulc(Lam[0], 1.7357142857142858)))))))); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, 0.048214285714285716, k); } y[16] = Ops::fma3(k, x[18], y[16]); y[18] = Ops::fma3(k, x[16], y[18]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[8], 1.7357142857142858, Ops::fmac(Lam[7], 1.7357142857142858, Ops::fmac(Lam[6], 1.7357142857142858, Ops::fmac(Lam[5], 1.7357142857142858, Ops::fmac(Lam[4], 1.7357142857142858, Ops::fmac(Lam[3], 3.4714285714285715, Ops::fmac(Lam[2], 1.7357142857142858, Ops::mulc(Lam[1], 1.7357142857142858)))))))); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, 0.048214285714285716, k); } y[16] = Ops::fma3(k, x[19], y[16]); y[19] = Ops::fma3(k, x[16], y[19]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[9], 3.4714285714285715, Ops::fmac(Lam[6], 3.4714285714285715, Ops::fmac(Lam[4], 3.4714285714285715, Ops::fmac(Lam[3], 3.4714285714285715, Ops::fmac(Lam[1], 3.4714285714285715, Ops::mulc(Lam[0], 3.4714285714285715)))))); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, 0.09642857142857143, k); } y[17] = Ops::fma3(k, x[17], y[17]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[9], 1.7357142857142858, Ops::fmac(Lam[8], 1.7357142857142858, Ops::fmac(Lam[6], 1.7357142857142858, Ops::fmac(Lam[5], 3.4714285714285715, Ops::fmac(Lam[3], 1.7357142857142858, Ops::fmac(Lam[2], 1.7357142857142858, Ops::fmac(Lam[1], 1.7357142857142858, Ops::mulc(Lam[0], 1.7357142857142858)))))))); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, 0.048214285714285716, k); } y[17] = Ops::fma3(k, x[18], y[17]); y[18] = Ops::fma3(k, x[17], y[18]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[9], 1.7357142857142858, Ops::fmac(Lam[8], 1.7357142857142858, Ops::fmac(Lam[6], 1.7357142857142858, Ops::fmac(Lam[5], 1.7357142857142858, Ops::fmac(Lam[4], 1.7357142857142858, Ops::fmac(Lam[3], 1.7357142857142858, Ops::fmac(Lam[2], 3.4714285714285715, Ops::mulc(Lam[1], 1.7357142857142858)))))))); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, 0.048214285714285716, k); } y[17] = Ops::fma3(k, x[19], y[17]); y[19] = Ops::fma3(k, x[17], y[19]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[9], 3.4714285714285715, Ops::fmac(Lam[8], 3.4714285714285715, Ops::fmac(Lam[7], 3.4714285714285715, Ops::fmac(Lam[3], 3.4714285714285715, Ops::fmac(Lam[2], 3.4714285714285715, Ops::mulc(Lam[0], 3.4714285714285715)))))); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, 0.09642857142857143, k); } y[18] = Ops::fma3(k, x[18], y[18]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[9], 1.7357142857142858, Ops::fmac(Lam[8], 1.7357142857142858, Ops::fmac(Lam[7], 1.7357142857142858, Ops::fmac(Lam[6], 1.7357142857142858, Ops::fmac(Lam[5], 1.7357142857142858, Ops::fmac(Lam[3], 1.7357142857142858, Ops::fmac(Lam[2], 1.7357142857142858, Ops::mulc(Lam[1], 3.4714285714285715)))))))); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, 0.048214285714285716, k); } y[18] = Ops::fma3(k, x[19], y[18]); y[19] = Ops::fma3(k, x[18], y[19]); }
    { if constexpr (STIFF) { k = Ops::fmac(Lam[9], 3.4714285714285715, Ops::fmac(Lam[8], 3.4714285714285715, Ops::fmac(Lam[7], 3.4714285714285715, Ops::fmac(Lam[6], 3.4714285714285715, Ops::fmac(Lam[5], 3.4714285714285715, Ops::mulc(Lam[4], 3.4714285714285715)))))); } else { k = Ops::zero(); } if constexpr (MASS) { k = Ops::fmac(vol, 0.09642857142857143, k); } y[19] = Ops::fma3(k, x[19], y[19]); }
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
