// Vertex-form stencil helpers shared by the finest-level kernels (fine.cu, fine_gs.cu).
// Vertex form of K u (Eq. 13): incident element t = a + 2b + 4c of vertex v has origin
// v - (1,1,1) + (a,b,c) and v is its local vertex 7 - t. The 3x3 coupling block between v
// and its neighbour v + d is
//     A_d = sum over (t, j) with bits(t) + bits(j) - 1 = d of E_t * K0[7 - t, j].
#pragma once

#include "dev_common.cuh"

namespace homo {

__device__ __forceinline__ void load_E8(const float* __restrict__ E, const Nb& nb, float (&Et)[8]) {
#pragma unroll
  for (int t = 0; t < 8; ++t) Et[t] = __ldg(E + nb.X[t & 1] + nb.Y[(t >> 1) & 1] + nb.Z[t >> 2]);
}

// 3x3 block A_d for neighbour offset (dx,dy,dz). Reflecting the cube through its centre
// planes maps any local vertex i to vertex 0 and negates the reflected displacement
// components, so K0[i][j] = R_i K0[0][i ^ j] R_i with R_i = diag(+-1) (-1 where bit k of
// i is set). In A_d every contributing element t has i ^ j = |d| (componentwise), hence
//   A_d[r][c] = K0[0][|d|][r][c] * sum_(t contributing) E_t s_r(t) s_c(t)   (s_r s_c = 1 if r = c),
// with s_k = d_k on axes where d_k != 0 and s_k = +1 / -1 for elements on the + / - side
// of v along axes where d_k = 0. So each block is 9 products with signed sums of the 8
// moduli instead of 9 FMAs per contributing element. All index and sign arithmetic folds
// at compile time once the callers' loops over d are unrolled.
__device__ __forceinline__ void nb_block(const KeParam& K, const float (&Et)[8], int dx, int dy,
                                         int dz, float (&A)[9]) {
  const int D[3] = {dx, dy, dz};
  const int m = (dx != 0 ? 1 : 0) + (dy != 0 ? 2 : 0) + (dz != 0 ? 4 : 0);
  float s0 = 0.f, s01 = 0.f, s02 = 0.f, s12 = 0.f;
#pragma unroll
  for (int t = 0; t < 8; ++t) {
    const int tb[3] = {t & 1, (t >> 1) & 1, t >> 2};
    bool in = true;
    int sg[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      if ((D[k] == 1 && tb[k] != 1) || (D[k] == -1 && tb[k] != 0)) in = false;
      sg[k] = D[k] != 0 ? D[k] : (tb[k] ? 1 : -1);
    }
    if (!in) continue;
    s0 += Et[t];
    s01 += sg[0] * sg[1] > 0 ? Et[t] : -Et[t];
    s02 += sg[0] * sg[2] > 0 ? Et[t] : -Et[t];
    s12 += sg[1] * sg[2] > 0 ? Et[t] : -Et[t];
  }
  const float* C = K.k + 3 * m;   // row r of K0[0][m] starts at K.k[r * 24 + 3 m]
  A[0] = C[0] * s0;       A[1] = C[1] * s01;      A[2] = C[2] * s02;
  A[3] = C[24] * s01;     A[4] = C[25] * s0;      A[5] = C[26] * s12;
  A[6] = C[48] * s02;     A[7] = C[49] * s12;     A[8] = C[50] * s0;
}

// Two FP32 lanes in one 64-bit register pair, for the two-lane FMA of sm_100 and later
// (fma.rn.f32x2): each lane is rounded exactly like a scalar fmaf, so a pair of load
// cases advanced together gives bitwise the result of two scalar chains in the same order.
typedef unsigned long long f32x2;

__device__ __forceinline__ f32x2 pack2(float lo, float hi) {
  f32x2 r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
  return r;
}

__device__ __forceinline__ void unpack2(f32x2 p, float& lo, float& hi) {
  asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(p));
}

// d = a * b + c per lane
__device__ __forceinline__ f32x2 ffma2(f32x2 a, f32x2 b, f32x2 c) {
  f32x2 d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
  return d;
}

__device__ __forceinline__ f32x2 fsub2(f32x2 a, f32x2 b) {
  f32x2 d;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}

__device__ __forceinline__ f32x2 fadd2(f32x2 a, f32x2 b) {
  f32x2 d;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}

// Solve the SPD 3x3 system S y = b for NC right-hand sides (LDL^T, FP32).
template <int NC>
__device__ __forceinline__ void solve3xn(const float (&S)[9], float (&b)[3 * NC]) {
  const float d0 = S[0];
  const float l10 = S[3] / d0, l20 = S[6] / d0;
  const float d1 = S[4] - l10 * S[1];
  const float l21 = (S[7] - l20 * S[1]) / d1;
  const float d2 = S[8] - l20 * S[2] - l21 * (S[5] - l10 * S[2]);
  const float i0 = 1.f / d0, i1 = 1.f / d1, i2 = 1.f / d2;
#pragma unroll
  for (int c = 0; c < NC; ++c) {
    float y0 = b[3 * c], y1 = b[3 * c + 1], y2 = b[3 * c + 2];
    y1 -= l10 * y0;
    y2 -= l20 * y0 + l21 * y1;
    float x2 = y2 * i2;
    float x1 = y1 * i1 - l21 * x2;
    float x0 = y0 * i0 - l10 * x1 - l20 * x2;
    b[3 * c] = x0;
    b[3 * c + 1] = x1;
    b[3 * c + 2] = x2;
  }
}

__device__ __forceinline__ void solve3x6(const float (&S)[9], float (&b)[18]) { solve3xn<kCases>(S, b); }

}  // namespace homo
