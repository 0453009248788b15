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

// 3x3 block A_d for neighbour offset (dx,dy,dz); all index arithmetic folds at compile
// time once the callers' loops are unrolled.
__device__ __forceinline__ void nb_block(const KeParam& K, const float (&Et)[8], int dx, int dy,
                                         int dz, float (&A)[9]) {
#pragma unroll
  for (int q = 0; q < 9; ++q) A[q] = 0.f;
#pragma unroll
  for (int t = 0; t < 8; ++t) {
    const int ja = dx + 1 - (t & 1), jb = dy + 1 - ((t >> 1) & 1), jc = dz + 1 - (t >> 2);
    if (ja < 0 || ja > 1 || jb < 0 || jb > 1 || jc < 0 || jc > 1) continue;
    const int j = ja + 2 * jb + 4 * jc, row = 7 - t;
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
      for (int c = 0; c < 3; ++c)
        A[3 * r + c] = fmaf(Et[t], K.k[(3 * row + r) * 24 + 3 * j + c], A[3 * r + c]);
  }
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
