// One colour pass of the finest-level 8-colour block Gauss-Seidel smoother (Eq. 15-16).
#include "stencil.cuh"

namespace homo {

namespace {

// One colour pass of 8-colour block Gauss-Seidel (Eq. 15-16): for every vertex v of
// the colour, S_v u_v = f_v - M_v with S_v = A_0 and M_v = sum_(d != 0) A_d u_(v+d).
// The neighbour v + d has colour (colour XOR oddness-mask of d), never the pass's own
// colour, so its value is not written during the pass (read through the read-only
// path). first != 0: first sweep from u = 0 in colour order 0..7, where neighbours of a
// higher colour still hold zero and are skipped (u need not be cleared beforehand).
// The load cases are split over blockIdx.y in groups of CASES (3: the blocks A_d are
// rebuilt per group, which keeps registers low and puts more loads in flight; 6: built
// once). Every variant (CASES, BLOCK) performs the same arithmetic per vertex and case in
// the same order, so all give bitwise the same result; homo_autotune picks the fastest
// for a grid size.
template <int CASES, int BLOCK>
__global__ void __launch_bounds__(BLOCK, (CASES == 3 ? 1024 : 512) / BLOCK)
    k_fine_gs(const __grid_constant__ KeParam K, const float* __restrict__ E, const float* __restrict__ f,
              float* __restrict__ u, int n, int colour, int first, const double* __restrict__ fmean) {
  constexpr int kGsCases = CASES;
  const size_t N = static_cast<size_t>(n) * n * n;
  const int h = n >> 1;
  const size_t Nh = static_cast<size_t>(h) * h * h;
  const int cx = colour & 1, cy = (colour >> 1) & 1, cz = colour >> 2;
  const int q0 = 3 * kGsCases * blockIdx.y;                // first plane of the case group
  for (size_t m = static_cast<size_t>(blockIdx.x) * blockDim.x + threadIdx.x; m < Nh;
       m += static_cast<size_t>(gridDim.x) * blockDim.x) {
    int i, j, k;
    decode3(static_cast<unsigned>(m), static_cast<unsigned>(h), i, j, k);
    const int x = 2 * i + cx, y = 2 * j + cy, z = 2 * k + cz;
    const size_t v = static_cast<size_t>(x) + static_cast<size_t>(n) * (y + static_cast<size_t>(n) * z);
    const Nb nb = make_nb(x, y, z, n);
    float Et[8];
    load_E8(E, nb, Et);
    // The cases advance in pairs (c, c + 1) on the two lanes of f32x2 registers: pair
    // p holds cases 2p and 2p + 1, a lone last case (CASES = 3) runs in scalar FMAs.
    constexpr int kPairs = kGsCases / 2;
    constexpr bool kOdd = (kGsCases & 1) != 0;
    f32x2 rp[3 * kPairs];
    float rs[3];
#pragma unroll
    for (int p = 0; p < kPairs; ++p)
#pragma unroll
      for (int r = 0; r < 3; ++r) {
        const int qa = 3 * (2 * p) + r, qb = qa + 3;
        rp[3 * p + r] = pack2(__ldg(f + (q0 + qa) * N + v) - (fmean ? static_cast<float>(fmean[q0 + qa]) : 0.f),
                              __ldg(f + (q0 + qb) * N + v) - (fmean ? static_cast<float>(fmean[q0 + qb]) : 0.f));
      }
    if (kOdd) {
#pragma unroll
      for (int r = 0; r < 3; ++r) {
        const int q = 3 * (kGsCases - 1) + r;
        rs[r] = __ldg(f + (q0 + q) * N + v) - (fmean ? static_cast<float>(fmean[q0 + q]) : 0.f);
      }
    }
#pragma unroll
    for (int d = 0; d < 27; ++d) {
      if (d == 13) continue;
      const int dx = d % 3 - 1, dy = (d / 3) % 3 - 1, dz = d / 9 - 1;
      const int odd = (dx != 0) | ((dy != 0) << 1) | ((dz != 0) << 2);
      if (first && (colour ^ odd) > colour) continue;
      float A[9];
      nb_block(K, Et, dx, dy, dz, A);
      f32x2 nA[9];
#pragma unroll
      for (int e = 0; e < 9; ++e) nA[e] = pack2(-A[e], -A[e]);
      const size_t w = static_cast<size_t>(nb.X[dx + 1] + nb.Y[dy + 1] + nb.Z[dz + 1]);
      const float* ur = u + q0 * N + w;
#pragma unroll
      for (int p = 0; p < kPairs; ++p) {
        f32x2 uu[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) uu[k] = pack2(__ldg(ur + (6 * p + k) * N), __ldg(ur + (6 * p + 3 + k) * N));
#pragma unroll
        for (int r = 0; r < 3; ++r)
          rp[3 * p + r] = ffma2(nA[3 * r + 2], uu[2], ffma2(nA[3 * r + 1], uu[1], ffma2(nA[3 * r], uu[0], rp[3 * p + r])));
      }
      if (kOdd) {
        const int c = kGsCases - 1;
        const float u0 = __ldg(ur + (3 * c) * N), u1 = __ldg(ur + (3 * c + 1) * N),
                    u2 = __ldg(ur + (3 * c + 2) * N);
#pragma unroll
        for (int r = 0; r < 3; ++r)
          rs[r] = fmaf(-A[3 * r + 2], u2, fmaf(-A[3 * r + 1], u1, fmaf(-A[3 * r], u0, rs[r])));
      }
    }
    float rhs[3 * kGsCases];
#pragma unroll
    for (int p = 0; p < kPairs; ++p)
#pragma unroll
      for (int r = 0; r < 3; ++r) unpack2(rp[3 * p + r], rhs[3 * (2 * p) + r], rhs[3 * (2 * p + 1) + r]);
    if (kOdd) {
#pragma unroll
      for (int r = 0; r < 3; ++r) rhs[3 * (kGsCases - 1) + r] = rs[r];
    }
    float S[9];
    nb_block(K, Et, 0, 0, 0, S);
    solve3xn<kGsCases>(S, rhs);
#pragma unroll
    for (int q = 0; q < 3 * kGsCases; ++q) u[(q0 + q) * N + v] = rhs[q];
  }
}

template <int CASES, int BLOCK>
cudaError_t gs_launch(const homo_ctx* c, int colour, const float* f, float* u, int first, const double* fmean) {
  const size_t h = static_cast<size_t>(c->n / 2);
  const dim3 grid(grid_for(h * h * h, BLOCK), kCases / CASES);
  k_fine_gs<CASES, BLOCK><<<grid, BLOCK, 0, c->stream>>>(c->ke, c->E, f, u, c->n, colour, first, fmean);
  return cudaGetLastError();
}

}  // namespace

bool gs_variant_ok(int cases, int block) { return (cases == 3 || cases == 6) && (block == 128 || block == 256); }

cudaError_t launch_fine_gs(const homo_ctx* c, int colour, const float* f, float* u, int first,
                           const double* fmean) {
  if (c->gs_cases == 6)
    return c->gs_block == 128 ? gs_launch<6, 128>(c, colour, f, u, first, fmean)
                              : gs_launch<6, 256>(c, colour, f, u, first, fmean);
  return c->gs_block == 128 ? gs_launch<3, 128>(c, colour, f, u, first, fmean)
                            : gs_launch<3, 256>(c, colour, f, u, first, fmean);
}

}  // namespace homo
