// Coarse levels of the multigrid hierarchy (Sec. 3.3, Sec. 4.2): Galerkin stencils,
// stored-stencil relaxation and residual, trilinear transfers and the direct coarsest
// solve with the rigid-translation null space projected out.
#include "dev_common.cuh"

#include <algorithm>
#include <mutex>

namespace homo {

namespace {

struct BfParam {
  float b[8 * 576];   // B_f = P_f^T K0 P_f for the 8 fine elements of a coarse element
};

// Level-1 stencil from the fine moduli (Eq. 17-18, grouped per coarse element): the
// coarse element with origin O has matrix sum_f E[2O + f] B_f; vertex V is local vertex
// 7 - t of its incident coarse element t, and local vertex J of that element is the
// neighbour V + bits(t) + bits(J) - 1. One thread per coarse vertex.
__global__ void __launch_bounds__(128) k_level1(const __grid_constant__ BfParam B,
                                                const float* __restrict__ E, int nf,
                                                float* __restrict__ st, int nc, bool cb) {
  const size_t Nc = static_cast<size_t>(nc) * nc * nc;
  for (size_t p = static_cast<size_t>(blockIdx.x) * blockDim.x + threadIdx.x; p < Nc;
       p += static_cast<size_t>(gridDim.x) * blockDim.x) {
    int X, Y, Z;
    vertex_of_pos(p, nc, cb, X, Y, Z);
    // fine elements of the 4x4x4 box with origin 2V - (2,2,2)
    float Eb[64];
    int ix[4], iy[4], iz[4];
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      ix[a] = ((2 * X - 2 + a) % nf + nf) % nf;
      iy[a] = (((2 * Y - 2 + a) % nf + nf) % nf) * nf;
      iz[a] = (((2 * Z - 2 + a) % nf + nf) % nf) * nf * nf;
    }
#pragma unroll
    for (int c = 0; c < 4; ++c)
#pragma unroll
      for (int b = 0; b < 4; ++b)
#pragma unroll
        for (int a = 0; a < 4; ++a) Eb[a + 4 * b + 16 * c] = __ldg(E + ix[a] + iy[b] + iz[c]);
#pragma unroll 1
    for (int d = 0; d < 27; ++d) {
      const int dx = d % 3 - 1, dy = (d / 3) % 3 - 1, dz = d / 9 - 1;
      float A[9];
#pragma unroll
      for (int q = 0; q < 9; ++q) A[q] = 0.f;
#pragma unroll
      for (int t = 0; t < 8; ++t) {
        const int ta = t & 1, tb = (t >> 1) & 1, tc = t >> 2;
        const int Ja = dx + 1 - ta, Jb = dy + 1 - tb, Jc = dz + 1 - tc;
        if (Ja < 0 || Ja > 1 || Jb < 0 || Jb > 1 || Jc < 0 || Jc > 1) continue;
        const int J = Ja + 2 * Jb + 4 * Jc, row = 7 - t;
#pragma unroll
        for (int f = 0; f < 8; ++f) {
          const float Ef = Eb[(2 * ta + (f & 1)) + 4 * (2 * tb + ((f >> 1) & 1)) + 16 * (2 * tc + (f >> 2))];
#pragma unroll
          for (int r = 0; r < 3; ++r)
#pragma unroll
            for (int c = 0; c < 3; ++c)
              A[3 * r + c] = fmaf(Ef, B.b[f * 576 + (3 * row + r) * 24 + 3 * J + c], A[3 * r + c]);
        }
      }
#pragma unroll
      for (int q = 0; q < 9; ++q) st[static_cast<size_t>(9 * d + q) * Nc + p] = A[q];
    }
  }
}

// One axis of the Galerkin product R K I (Eq. 17-18 on coarse levels). The trilinear
// transfers are tensor products of the 1-D linear interpolation, so R K I factors into
// three one-axis coarsenings, each a 27-point block stencil again. Coarsening axis `ax`
// of a stencil S on an (mx, my, mz) grid: for output vertex V and output offset d,
//   S'(V, d) = sum over a, e in {-1,0,1} with |2 d_ax + e - a| <= 1 of
//              w(a) w(e) S(V with x_ax -> 2 V_ax + a, d with d_ax -> 2 d_ax + e - a),
// w(t) = 1 - |t|/2: 7 pairs when d_ax = 0, 3 when d_ax = +-1. src_cb / dst_cb: the grid
// is cubic and its stencil planes are colour-blocked (a level's own layout); otherwise
// x-fastest. Thread per (d, output vertex).
template <int ax>
__global__ void __launch_bounds__(256) k_galerkin_axis(const float* __restrict__ src, int mx, int my, int mz,
                                                       bool src_cb, float* __restrict__ dst, bool dst_cb) {
  const int ox = ax == 0 ? mx / 2 : mx, oy = ax == 1 ? my / 2 : my, oz = ax == 2 ? mz / 2 : mz;
  const size_t Nin = static_cast<size_t>(mx) * my * mz;
  const size_t Nout = static_cast<size_t>(ox) * oy * oz;
  const size_t total = 27 * Nout;
  for (size_t it = static_cast<size_t>(blockIdx.x) * blockDim.x + threadIdx.x; it < total;
       it += static_cast<size_t>(gridDim.x) * blockDim.x) {
    const int d = static_cast<int>(it / Nout);
    const size_t p = it - static_cast<size_t>(d) * Nout;
    int V[3];
    if (dst_cb) {
      vertex_of_pos(p, ox, true, V[0], V[1], V[2]);
    } else {
      const unsigned q = static_cast<unsigned>(p) / static_cast<unsigned>(ox);
      V[0] = static_cast<int>(static_cast<unsigned>(p) - q * static_cast<unsigned>(ox));
      V[2] = static_cast<int>(q / static_cast<unsigned>(oy));
      V[1] = static_cast<int>(q - static_cast<unsigned>(V[2]) * static_cast<unsigned>(oy));
    }
    const int D[3] = {d % 3 - 1, (d / 3) % 3 - 1, d / 9 - 1};
    const int m_ax = ax == 0 ? mx : (ax == 1 ? my : mz);
    float A[9];
#pragma unroll
    for (int q = 0; q < 9; ++q) A[q] = 0.f;
#pragma unroll
    for (int a = -1; a <= 1; ++a) {
      int F[3] = {V[0], V[1], V[2]};
      int fa = 2 * V[ax] + a;
      fa = fa < 0 ? fa + m_ax : (fa >= m_ax ? fa - m_ax : fa);
      F[ax] = fa;
      const size_t pin = src_cb ? stencil_pos(F[0], F[1], F[2], mx, true)
                                : static_cast<size_t>(F[0]) + static_cast<size_t>(mx) *
                                      (F[1] + static_cast<size_t>(my) * F[2]);
      const float wa = a ? 0.5f : 1.f;
#pragma unroll
      for (int e = -1; e <= 1; ++e) {
        const int bax = 2 * D[ax] + e - a;
        if (bax < -1 || bax > 1) continue;
        int B[3] = {D[0], D[1], D[2]};
        B[ax] = bax;
        const int dd = (B[0] + 1) + 3 * (B[1] + 1) + 9 * (B[2] + 1);
        const float ww = wa * (e ? 0.5f : 1.f);
#pragma unroll
        for (int q = 0; q < 9; ++q) A[q] = fmaf(ww, __ldg(src + static_cast<size_t>(9 * dd + q) * Nin + pin), A[q]);
      }
    }
#pragma unroll
    for (int q = 0; q < 9; ++q) dst[static_cast<size_t>(9 * d + q) * Nout + p] = A[q];   // p: output position
  }
}

// Stencil entry as FP32 from FP32 or BF16 storage.
__device__ __forceinline__ float ld_st(const float* p) { return __ldg(p); }
__device__ __forceinline__ float ld_st(const __nv_bfloat16* p) { return __bfloat162float(__ldg(p)); }

// Mixed precision: st16 = BF16 of (A_d(v) + A_-d(v+d)^T) / 2 for every vertex v and
// neighbour d. Both partners of a pair are formed from the same two FP32 blocks (FP32
// addition commutes and the halving is exact), so the rounded operator is exactly
// symmetric. Thread per (d, position); writes the BF16 plane layout of st.
__global__ void __launch_bounds__(256) k_stencil_bf16(const float* __restrict__ st, int n, bool cb,
                                                      __nv_bfloat16* __restrict__ st16) {
  const size_t N = static_cast<size_t>(n) * n * n;
  const size_t total = 27 * N;
  for (size_t it = static_cast<size_t>(blockIdx.x) * blockDim.x + threadIdx.x; it < total;
       it += static_cast<size_t>(gridDim.x) * blockDim.x) {
    const int d = static_cast<int>(it / N);
    const size_t p = it - static_cast<size_t>(d) * N;
    int X, Y, Z;
    vertex_of_pos(p, n, cb, X, Y, Z);
    const int dx = d % 3 - 1, dy = (d / 3) % 3 - 1, dz = d / 9 - 1;
    const int Xn = (X + dx + n) % n, Yn = (Y + dy + n) % n, Zn = (Z + dz + n) % n;
    const size_t pn = stencil_pos(Xn, Yn, Zn, n, cb);
    const int dm = 26 - d;                      // offset -d seen from the neighbour
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const float a = st[static_cast<size_t>(9 * d + 3 * r + c) * N + p];
        const float b = st[static_cast<size_t>(9 * dm + 3 * c + r) * N + pn];
        st16[static_cast<size_t>(9 * d + 3 * r + c) * N + p] = __float2bfloat16_rn(0.5f * (a + b));
      }
  }
}

// LDL^T factors of the symmetric 3x3 diagonal block S_v (Eq. 16): multipliers l10, l20,
// l21 and the reciprocal pivots i0, i1, i2.
struct Factor3 {
  float l10, l20, l21, i0, i1, i2;
};

__device__ __forceinline__ Factor3 factor3(const float (&S)[9]) {
  Factor3 F;
  const float d0 = S[0];
  F.l10 = S[3] / d0;
  F.l20 = S[6] / d0;
  const float d1 = S[4] - F.l10 * S[1];
  F.l21 = (S[7] - F.l20 * S[1]) / d1;
  const float d2 = S[8] - F.l20 * S[2] - F.l21 * (S[5] - F.l10 * S[2]);
  F.i0 = 1.f / d0;
  F.i1 = 1.f / d1;
  F.i2 = 1.f / d2;
  return F;
}

// Solve S_v x = (y0, y1, y2) in place for one load case.
__device__ __forceinline__ void solve3(const Factor3& F, float& y0, float& y1, float& y2) {
  y1 -= F.l10 * y0;
  y2 -= F.l20 * y0 + F.l21 * y1;
  const float x2 = y2 * F.i2;
  const float x1 = y1 * F.i1 - F.l21 * x2;
  const float x0 = y0 * F.i0 - F.l10 * x1 - F.l20 * x2;
  y0 = x0;
  y1 = x1;
  y2 = x2;
}

__device__ __forceinline__ void solve3x6c(const float (&S)[9], float (&b)[18]) {
  const Factor3 F = factor3(S);
#pragma unroll
  for (int c = 0; c < kCases; ++c) solve3(F, b[3 * c], b[3 * c + 1], b[3 * c + 2]);
}

// One colour pass of block Gauss-Seidel (Eq. 15-16) with the stored stencil. Neighbours
// have other colours and are not written during the pass. first != 0: first sweep from
// x = 0 in colour order 0..7 (higher-colour neighbours are still zero and skipped).
template <typename T>
__global__ void __launch_bounds__(256) k_coarse_gs(const T* __restrict__ st,
                                                   const float* __restrict__ f,
                                                   float* __restrict__ x, int n, int colour,
                                                   int first) {
  const size_t N = static_cast<size_t>(n) * n * n;
  const int h = n >> 1;
  const size_t Nh = static_cast<size_t>(h) * h * h;
  const int cx = colour & 1, cy = (colour >> 1) & 1, cz = colour >> 2;
  for (size_t m = static_cast<size_t>(blockIdx.x) * blockDim.x + threadIdx.x; m < Nh;
       m += static_cast<size_t>(gridDim.x) * blockDim.x) {
    int i, j, k;
    decode3(static_cast<unsigned>(m), static_cast<unsigned>(h), i, j, k);
    const int X = 2 * i + cx, Y = 2 * j + cy, Z = 2 * k + cz;
    const size_t p = static_cast<size_t>(colour) * Nh + m;
    const size_t v = static_cast<size_t>(X) + static_cast<size_t>(n) * (Y + static_cast<size_t>(n) * Z);
    const Nb nb = make_nb(X, Y, Z, n);
    float rhs[kPlanes];
#pragma unroll
    for (int q = 0; q < kPlanes; ++q) rhs[q] = __ldg(f + q * N + v);
    float S[9];
#pragma unroll
    for (int q = 0; q < 9; ++q) S[q] = ld_st(st + static_cast<size_t>(9 * 13 + q) * N + p);
#pragma unroll
    for (int d = 0; d < 27; ++d) {
      if (d == 13) continue;
      const int dx = d % 3 - 1, dy = (d / 3) % 3 - 1, dz = d / 9 - 1;
      const int odd = (dx != 0) | ((dy != 0) << 1) | ((dz != 0) << 2);
      if (first && (colour ^ odd) > colour) continue;
      float A[9];
#pragma unroll
      for (int q = 0; q < 9; ++q) A[q] = ld_st(st + static_cast<size_t>(9 * d + q) * N + p);
      const size_t w = static_cast<size_t>(nb.X[dx + 1] + nb.Y[dy + 1] + nb.Z[dz + 1]);
      const float* xr = x;
#pragma unroll
      for (int c = 0; c < kCases; ++c) {
        const float u0 = __ldg(xr + (3 * c) * N + w), u1 = __ldg(xr + (3 * c + 1) * N + w),
                    u2 = __ldg(xr + (3 * c + 2) * N + w);
#pragma unroll
        for (int r = 0; r < 3; ++r)
          rhs[3 * c + r] = fmaf(-A[3 * r + 2], u2, fmaf(-A[3 * r + 1], u1, fmaf(-A[3 * r], u0, rhs[3 * c + r])));
      }
    }
    solve3x6c(S, rhs);
#pragma unroll
    for (int q = 0; q < kPlanes; ++q) x[q * N + v] = rhs[q];
  }
}

// One load case of one vertex of a block Gauss-Seidel colour pass (Eq. 15-16): exactly
// the arithmetic of that case in k_coarse_gs (the same FMAs in the same order, the same
// factorisation and solve), so it produces bitwise the same value. The 26 neighbours are
// visited in three z-layers of 9 (d = 0..8, 9..17, 18..26, the order of the FMA chain);
// the 108 stencil and displacement values of a layer are loaded before its FMAs, so a
// thread waits for three rounds of loads instead of one per neighbour (the small coarse
// levels are bound by that latency). COHERENT: x is read through L2 only, for kernels in
// which other CTAs write x between colour passes; otherwise through the read-only path
// (a pass reads only vertices of other colours, which it does not write).
template <typename T, bool COHERENT>
__device__ __forceinline__ void gs_item(const T* __restrict__ st, const float* __restrict__ f, float* x,
                                        int n, size_t N, unsigned Nh, int h, int colour, int fz, int c,
                                        unsigned m) {
  const int cx = colour & 1, cy = (colour >> 1) & 1, cz = colour >> 2;
  int i, j, kk;
  decode3(m, static_cast<unsigned>(h), i, j, kk);
  const int X = 2 * i + cx, Y = 2 * j + cy, Z = 2 * kk + cz;
  const size_t p = static_cast<size_t>(colour) * Nh + m;
  const size_t v = static_cast<size_t>(X) + static_cast<size_t>(n) * (Y + static_cast<size_t>(n) * Z);
  const Nb nb = make_nb(X, Y, Z, n);
  const float* fc = f + static_cast<size_t>(3 * c) * N;
  const float* xc = x + static_cast<size_t>(3 * c) * N;
  float b0 = __ldg(fc + v), b1 = __ldg(fc + N + v), b2 = __ldg(fc + 2 * N + v);
  float S[9];
#pragma unroll
  for (int layer = 0; layer < 3; ++layer) {
    float A[9][9], U[9][3];
#pragma unroll
    for (int e = 0; e < 9; ++e) {
      const int d = 9 * layer + e;
      const int dx = d % 3 - 1, dy = (d / 3) % 3 - 1, dz = d / 9 - 1;
      const int odd = (dx != 0) | ((dy != 0) << 1) | ((dz != 0) << 2);
      if (d == 13) {
#pragma unroll
        for (int q = 0; q < 9; ++q) S[q] = ld_st(st + static_cast<size_t>(9 * 13 + q) * N + p);
        continue;
      }
      if (fz && (colour ^ odd) > colour) continue;
#pragma unroll
      for (int q = 0; q < 9; ++q) A[e][q] = ld_st(st + static_cast<size_t>(9 * d + q) * N + p);
      const size_t w = static_cast<size_t>(nb.X[dx + 1] + nb.Y[dy + 1] + nb.Z[dz + 1]);
      if (COHERENT) {
        U[e][0] = __ldcg(xc + w);
        U[e][1] = __ldcg(xc + N + w);
        U[e][2] = __ldcg(xc + 2 * N + w);
      } else {
        U[e][0] = __ldg(xc + w);
        U[e][1] = __ldg(xc + N + w);
        U[e][2] = __ldg(xc + 2 * N + w);
      }
    }
#pragma unroll
    for (int e = 0; e < 9; ++e) {
      const int d = 9 * layer + e;
      const int dx = d % 3 - 1, dy = (d / 3) % 3 - 1, dz = d / 9 - 1;
      const int odd = (dx != 0) | ((dy != 0) << 1) | ((dz != 0) << 2);
      if (d == 13 || (fz && (colour ^ odd) > colour)) continue;
      const float u0 = U[e][0], u1 = U[e][1], u2 = U[e][2];
      b0 = fmaf(-A[e][2], u2, fmaf(-A[e][1], u1, fmaf(-A[e][0], u0, b0)));
      b1 = fmaf(-A[e][5], u2, fmaf(-A[e][4], u1, fmaf(-A[e][3], u0, b1)));
      b2 = fmaf(-A[e][8], u2, fmaf(-A[e][7], u1, fmaf(-A[e][6], u0, b2)));
    }
  }
  solve3(factor3(S), b0, b1, b2);
  float* xo = x + static_cast<size_t>(3 * c) * N + v;
  if (COHERENT) {
    __stcg(xo, b0);
    __stcg(xo + N, b1);
    __stcg(xo + 2 * N, b2);
  } else {
    xo[0] = b0;
    xo[N] = b1;
    xo[2 * N] = b2;
  }
}

// Work items of a colour pass: one warp per (32 consecutive vertices of the colour, load
// case), the six case warps of a vertex block adjacent, so that a 192-thread CTA covers
// all six cases of its 32 vertices (their stencil rows are shared through L1) and every
// warp's loads are coalesced along the vertex index. Returns false for the padding lanes
// beyond the last vertex.
constexpr int kItemBlock = 192;

__device__ __forceinline__ bool gs_item_index(unsigned it, unsigned Nh, int& c, unsigned& m) {
  const unsigned g = it >> 5;
  const unsigned mb = g / kCases;
  c = static_cast<int>(g - mb * kCases);
  m = mb * 32 + (it & 31);
  return m < Nh;
}

__host__ __device__ inline unsigned gs_items(unsigned Nh) { return (Nh + 31) / 32 * 32 * kCases; }

// One colour pass with a thread per (load case, vertex of the colour): six times the
// threads of k_coarse_gs, each with a sixth of its FMAs and its loads in flight a z-layer
// at a time.
template <typename T>
__global__ void __launch_bounds__(kItemBlock) k_coarse_gs_item(const T* __restrict__ st,
                                                               const float* __restrict__ f, float* x,
                                                               int n, int colour, int first) {
  const size_t N = static_cast<size_t>(n) * n * n;
  const int h = n >> 1;
  const unsigned Nh = static_cast<unsigned>(h) * h * h;
  const unsigned items = gs_items(Nh);
  for (unsigned it = blockIdx.x * blockDim.x + threadIdx.x; it < items; it += gridDim.x * blockDim.x) {
    int c;
    unsigned m;
    if (gs_item_index(it, Nh, c, m)) gs_item<T, false>(st, f, x, n, N, Nh, h, colour, first, c, m);
  }
}

// Every sweep of one smoothing phase on a small level in one launch. Gauss-Seidel does
// not couple the load cases, so the grid is six thread-block clusters of csize CTAs, one
// per case, that never wait on one another: a cluster's colour passes are separated by
// its own hardware barrier (release at arrival, acquire at the wait, cluster scope), so a
// pass sees every value the passes before it wrote; x is read and written through L2.
// Spreading the cases over six clusters puts six times as many SMs on the small levels,
// whose passes are bound by load latency and load issue. Items as in k_coarse_gs_item
// (gs_item per vertex and case), so the iterates are bitwise those of the per-colour
// launches. sweeps >= 1; reverse: colours 7..0; first: the first sweep starts from x = 0
// (forward order only, as in k_coarse_gs).
__device__ __forceinline__ void cluster_barrier() {
  asm volatile("barrier.cluster.arrive.release;\n\tbarrier.cluster.wait.acquire;" ::: "memory");
}

constexpr int kClusterBlock = 256;

template <typename T>
__global__ void __launch_bounds__(kClusterBlock) k_coarse_gs_cluster(const T* __restrict__ st,
                                                                     const float* __restrict__ f,
                                                                     float* x, int n, int sweeps,
                                                                     int reverse, int first, int csize) {
  const size_t N = static_cast<size_t>(n) * n * n;
  const int h = n >> 1;
  const unsigned Nh = static_cast<unsigned>(h) * h * h;
  const int c = static_cast<int>(blockIdx.x) / csize;   // load case of this cluster
  const unsigned nthreads = static_cast<unsigned>(csize) * blockDim.x;
  const unsigned tid = (blockIdx.x - static_cast<unsigned>(c * csize)) * blockDim.x + threadIdx.x;
  for (int s = 0; s < sweeps; ++s) {
    const int fz = first && s == 0 && !reverse ? 1 : 0;
    for (int k = 0; k < 8; ++k) {
      const int colour = reverse ? 7 - k : k;
      for (unsigned m = tid; m < Nh; m += nthreads) gs_item<T, true>(st, f, x, n, N, Nh, h, colour, fz, c, m);
      cluster_barrier();
    }
  }
}

// ---- shared-memory-resident form of the small-level smoother
// Six clusters again, one per load case; the CTAs of a cluster split each colour's
// vertices into ranges of at most kResVerts (CTA r owns positions [r Mper, (r+1) Mper) of
// every colour, three threads per vertex, one per block row). Every CTA keeps a full copy of its case's
// displacement in shared memory, so all neighbour reads of a pass are shared-memory
// loads; the owner of a vertex writes its new value into every CTA's copy (distributed
// shared memory) before the cluster barrier that ends the pass. Each CTA streams the
// stencil rows of its own vertices for the next colour pass into a second buffer with
// asynchronous copies while the current pass computes, and keeps the right-hand side of
// its vertices for all colours. The arithmetic per vertex is gs_item's, on the same
// values in the same order: bitwise the iterates of the other forms.
constexpr int kResVerts = 64;     // vertices per colour per CTA, at most
constexpr int kResThreads = 256;  // threads per CTA: all stage, 3 x kResVerts compute (a row each)

__device__ __forceinline__ unsigned smem_addr(const void* p) {
  return static_cast<unsigned>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void cp_async_f4(float* dst, const float* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(smem_addr(dst)), "l"(src) : "memory");
}

__device__ __forceinline__ void cp_async_f16(float* dst, const float* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(smem_addr(dst)), "l"(src) : "memory");
}

// value into the same shared-memory offset of CTA `rank` of the cluster
__device__ __forceinline__ void st_cluster_f32(const float* local, unsigned rank, float v) {
  unsigned remote;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(remote) : "r"(smem_addr(local)), "r"(rank));
  asm volatile("st.shared::cluster.f32 [%0], %1;" ::"r"(remote), "f"(v) : "memory");
}

// Shared memory of k_coarse_gs_resident in floats: the case's displacement (3N), two
// stencil buffers (2 x 243 x Mper) and the owned right-hand sides (8 x 3 x Mper).
__host__ __device__ inline size_t resident_smem_floats(size_t N, int Mper) {
  return 3 * N + 2 * static_cast<size_t>(kStencil) * Mper + 24 * static_cast<size_t>(Mper);
}

// Stage the stencil rows of positions colour*Nh + m0 .. + mcount of every plane: 16-byte
// copies when every segment is 16-byte aligned (vec), 4-byte copies otherwise. Thread t
// copies chunk t % per of planes t / per, t / per + blockDim / per, ... (per = chunks per
// plane; the quotient is taken once per launch, not per copy).
struct StageMap {
  int per, plane0, step, chunk;   // step 0: the thread copies nothing
};

__device__ __forceinline__ StageMap stage_map(int mcount, bool vec) {
  StageMap m;
  m.per = vec ? (mcount >> 2) : mcount;
  const int planes_per_pass = m.per > 0 ? static_cast<int>(blockDim.x) / m.per : 0;
  if (planes_per_pass == 0 || static_cast<int>(threadIdx.x) >= planes_per_pass * m.per) {
    m.plane0 = 0;
    m.step = 0;
    m.chunk = 0;
    return m;
  }
  m.plane0 = static_cast<int>(threadIdx.x) / m.per;
  m.chunk = static_cast<int>(threadIdx.x) - m.plane0 * m.per;
  m.step = planes_per_pass;
  return m;
}

__device__ __forceinline__ void stage_rows(const float* __restrict__ st, size_t N, unsigned Nh, int colour,
                                           unsigned m0, int Mper, bool vec, const StageMap& sm_, float* buf) {
  if (sm_.step > 0) {
    const int j = vec ? (sm_.chunk << 2) : sm_.chunk;
    const float* src = st + static_cast<size_t>(colour) * Nh + m0 + j + static_cast<size_t>(sm_.plane0) * N;
    float* dst = buf + sm_.plane0 * Mper + j;
    const size_t src_step = static_cast<size_t>(sm_.step) * N;
    const int dst_step = sm_.step * Mper;
    for (int plane = sm_.plane0; plane < kStencil; plane += sm_.step, src += src_step, dst += dst_step) {
      if (vec) cp_async_f16(dst, src);
      else cp_async_f4(dst, src);
    }
  }
  asm volatile("cp.async.commit_group;\n" ::: "memory");
}

__global__ void __launch_bounds__(kResThreads) k_coarse_gs_resident(const float* __restrict__ st,
                                                                  const float* __restrict__ f, float* x,
                                                                  int n, int sweeps, int reverse, int first,
                                                                  int csize, int Mper, int vec16) {
  extern __shared__ float sm[];
  const size_t N = static_cast<size_t>(n) * n * n;
  const int h = n >> 1;
  const unsigned Nh = static_cast<unsigned>(h) * h * h;
  const int c = static_cast<int>(blockIdx.x) / csize;   // load case of this cluster
  const unsigned rank = blockIdx.x - static_cast<unsigned>(c * csize);
  const unsigned m0 = rank * static_cast<unsigned>(Mper);
  const int mcount = m0 >= Nh ? 0 : static_cast<int>(min(static_cast<unsigned>(Mper), Nh - m0));
  const bool vec = vec16 && (mcount % 4 == 0);   // vec16: st, N, Nh and Mper allow 16-byte segments
  float* us = sm;                                          // [3][N]
  float* sb[2] = {us + 3 * N, us + 3 * N + kStencil * Mper};
  float* fs = sb[1] + kStencil * Mper;                     // [8][3][Mper]
  const float* xc = x + static_cast<size_t>(3 * c) * N;
  const float* fc = f + static_cast<size_t>(3 * c) * N;
  const int r = static_cast<int>(threadIdx.x) / kResVerts;   // row of the vertex's block rows (3: stage only)
  const int j = static_cast<int>(threadIdx.x) - r * kResVerts;
  __shared__ float rows_s[3][kResVerts];

  for (size_t i = threadIdx.x; i < 3 * N; i += blockDim.x) us[i] = __ldcg(xc + i);
  for (int i = threadIdx.x; i < 8 * mcount; i += blockDim.x) {
    const int colour = i / mcount, jj = i - colour * mcount;
    int a, b, cc;
    decode3(m0 + jj, static_cast<unsigned>(h), a, b, cc);
    const size_t v = static_cast<size_t>(2 * a + (colour & 1)) +
                     static_cast<size_t>(n) * ((2 * b + ((colour >> 1) & 1)) + static_cast<size_t>(n) * (2 * cc + (colour >> 2)));
#pragma unroll
    for (int k = 0; k < 3; ++k) fs[(colour * 3 + k) * Mper + jj] = __ldg(fc + k * N + v);
  }
  const int total = sweeps * 8;
  const StageMap smap = stage_map(mcount, vec);
  stage_rows(st, N, Nh, reverse ? 7 : 0, m0, Mper, vec, smap, sb[0]);
  cluster_barrier();   // every copy of the displacement is loaded before any owner writes into it

  for (int pass = 0; pass < total; ++pass) {
    const int k = pass & 7;
    const int colour = reverse ? 7 - k : k;
    const int fz = first && pass < 8 && !reverse ? 1 : 0;
    if (pass + 1 < total) {
      const int kn = (pass + 1) & 7;
      stage_rows(st, N, Nh, reverse ? 7 - kn : kn, m0, Mper, vec, smap, sb[(pass + 1) & 1]);
    } else {
      asm volatile("cp.async.commit_group;\n" ::: "memory");
    }
    asm volatile("cp.async.wait_group 1;\n" ::: "memory");
    __syncthreads();
    // thread (row r, vertex j): the FMA chain of row r of the vertex's three rows (the
    // rows are independent chains); the solve gathers the three rows through rows_s
    const int cx = colour & 1, cy = (colour >> 1) & 1, cz = colour >> 2;
    size_t v = 0;
    if (r < 3 && j < mcount) {
      const float* S_ = sb[pass & 1];
      int a, b, cc;
      decode3(m0 + j, static_cast<unsigned>(h), a, b, cc);
      const int X = 2 * a + cx, Y = 2 * b + cy, Z = 2 * cc + cz;
      v = static_cast<size_t>(X) + static_cast<size_t>(n) * (Y + static_cast<size_t>(n) * Z);
      const Nb nb = make_nb(X, Y, Z, n);
      float br = fs[(colour * 3 + r) * Mper + j];
#pragma unroll
      for (int d = 0; d < 27; ++d) {
        if (d == 13) continue;
        const int dx = d % 3 - 1, dy = (d / 3) % 3 - 1, dz = d / 9 - 1;
        const int odd = (dx != 0) | ((dy != 0) << 1) | ((dz != 0) << 2);
        if (fz && (colour ^ odd) > colour) continue;
        const float* Ad = S_ + (9 * d + 3 * r) * Mper + j;
        const size_t w = static_cast<size_t>(nb.X[dx + 1] + nb.Y[dy + 1] + nb.Z[dz + 1]);
        br = fmaf(-Ad[2 * Mper], us[2 * N + w], fmaf(-Ad[Mper], us[N + w], fmaf(-Ad[0], us[w], br)));
      }
      rows_s[r][j] = br;
    }
    __syncthreads();
    if (r < 3 && j < mcount) {
      const float* S_ = sb[pass & 1];
      float S[9];
#pragma unroll
      for (int q = 0; q < 9; ++q) S[q] = S_[(9 * 13 + q) * Mper + j];
      float y0 = rows_s[0][j], y1 = rows_s[1][j], y2 = rows_s[2][j];
      solve3(factor3(S), y0, y1, y2);
      const float val = r == 0 ? y0 : (r == 1 ? y1 : y2);
      float* dst = us + static_cast<size_t>(r) * N + v;
      *dst = val;
      for (unsigned t = 0; t < static_cast<unsigned>(csize); ++t)
        if (t != rank) st_cluster_f32(dst, t, val);
    }
    cluster_barrier();
  }
  // every vertex is owned by one CTA: write the owned values back
  for (int i = threadIdx.x; i < 8 * mcount; i += blockDim.x) {
    const int colour = i / mcount, jj = i - colour * mcount;
    int a, b, cc;
    decode3(m0 + jj, static_cast<unsigned>(h), a, b, cc);
    const size_t v = static_cast<size_t>(2 * a + (colour & 1)) +
                     static_cast<size_t>(n) * ((2 * b + ((colour >> 1) & 1)) + static_cast<size_t>(n) * (2 * cc + (colour >> 2)));
    float* xo = x + static_cast<size_t>(3 * c) * N + v;
#pragma unroll
    for (int k = 0; k < 3; ++k) __stcg(xo + k * N, us[k * N + v]);
  }
}

// out = b - K x with the stored stencil; threads walk stencil positions (coalesced).
template <typename T>
__global__ void __launch_bounds__(256) k_coarse_residual(const T* __restrict__ st,
                                                         const float* __restrict__ b,
                                                         const float* __restrict__ x,
                                                         float* __restrict__ out, int n, bool cb) {
  const size_t N = static_cast<size_t>(n) * n * n;
  // vertices in lexicographic order: x, b and out are read and written in whole sectors;
  // with colour-blocked stencils a warp's stencil reads are two contiguous runs
  for (size_t v = static_cast<size_t>(blockIdx.x) * blockDim.x + threadIdx.x; v < N;
       v += static_cast<size_t>(gridDim.x) * blockDim.x) {
    int X, Y, Z;
    decode3(static_cast<unsigned>(v), static_cast<unsigned>(n), X, Y, Z);
    const size_t p = stencil_pos(X, Y, Z, n, cb);
    const Nb nb = make_nb(X, Y, Z, n);
    float acc[kPlanes];
#pragma unroll
    for (int q = 0; q < kPlanes; ++q) acc[q] = 0.f;
#pragma unroll
    for (int d = 0; d < 27; ++d) {
      const int dx = d % 3 - 1, dy = (d / 3) % 3 - 1, dz = d / 9 - 1;
      float A[9];
#pragma unroll
      for (int q = 0; q < 9; ++q) A[q] = ld_st(st + static_cast<size_t>(9 * d + q) * N + p);
      const size_t w = static_cast<size_t>(nb.X[dx + 1] + nb.Y[dy + 1] + nb.Z[dz + 1]);
#pragma unroll
      for (int c = 0; c < kCases; ++c) {
        const float u0 = __ldg(x + (3 * c) * N + w), u1 = __ldg(x + (3 * c + 1) * N + w),
                    u2 = __ldg(x + (3 * c + 2) * N + w);
#pragma unroll
        for (int r = 0; r < 3; ++r)
          acc[3 * c + r] = fmaf(A[3 * r], u0, fmaf(A[3 * r + 1], u1, fmaf(A[3 * r + 2], u2, acc[3 * c + r])));
      }
    }
#pragma unroll
    for (int q = 0; q < kPlanes; ++q) out[q * N + v] = __ldg(b + q * N + v) - acc[q];
  }
}

// Chebyshev step with the stored stencil (threads walk vertices in lexicographic order):
// mode 0: out = x_in + c0 S^-1 (b - K x_in); mode 1: out = x_in + c0 (x_in - out) +
// c1 S^-1 (b - K x_in), the previous iterate read from out and replaced in place.
// x_in == null stands for x_in = 0 (first step from zero). mode 2: out = S^-1 K x_in
// (power iteration for the largest eigenvalue of D^-1 K).
template <typename T>
__global__ void __launch_bounds__(256) k_coarse_cheb(const T* __restrict__ st,
                                                     const float* __restrict__ b,
                                                     const float* __restrict__ xin, float* out,
                                                     int n, bool cb, int mode, float c0, float c1) {
  const size_t N = static_cast<size_t>(n) * n * n;
  for (size_t v = static_cast<size_t>(blockIdx.x) * blockDim.x + threadIdx.x; v < N;
       v += static_cast<size_t>(gridDim.x) * blockDim.x) {
    int X, Y, Z;
    decode3(static_cast<unsigned>(v), static_cast<unsigned>(n), X, Y, Z);
    const size_t p = stencil_pos(X, Y, Z, n, cb);
    float acc[kPlanes];
#pragma unroll
    for (int q = 0; q < kPlanes; ++q) acc[q] = 0.f;
    if (xin) {
      const Nb nb = make_nb(X, Y, Z, n);
#pragma unroll
      for (int d = 0; d < 27; ++d) {
        const int dx = d % 3 - 1, dy = (d / 3) % 3 - 1, dz = d / 9 - 1;
        float A[9];
#pragma unroll
        for (int q = 0; q < 9; ++q) A[q] = ld_st(st + static_cast<size_t>(9 * d + q) * N + p);
        const size_t w = static_cast<size_t>(nb.X[dx + 1] + nb.Y[dy + 1] + nb.Z[dz + 1]);
#pragma unroll
        for (int c = 0; c < kCases; ++c) {
          const float u0 = __ldg(xin + (3 * c) * N + w), u1 = __ldg(xin + (3 * c + 1) * N + w),
                      u2 = __ldg(xin + (3 * c + 2) * N + w);
#pragma unroll
          for (int r = 0; r < 3; ++r)
            acc[3 * c + r] = fmaf(A[3 * r], u0, fmaf(A[3 * r + 1], u1, fmaf(A[3 * r + 2], u2, acc[3 * c + r])));
        }
      }
    }
    float S[9];
#pragma unroll
    for (int q = 0; q < 9; ++q) S[q] = ld_st(st + static_cast<size_t>(9 * 13 + q) * N + p);
    if (mode != 2) {
#pragma unroll
      for (int q = 0; q < kPlanes; ++q) acc[q] = __ldg(b + q * N + v) - acc[q];
    }
    solve3x6c(S, acc);
#pragma unroll
    for (int q = 0; q < kPlanes; ++q) {
      const size_t o = q * N + v;
      const float xc = xin ? __ldg(xin + o) : 0.f;
      if (mode == 0) out[o] = fmaf(c0, acc[q], xc);
      else if (mode == 1) out[o] = fmaf(c1, acc[q], fmaf(c0, xc - out[o], xc));
      else if (mode == 3) out[o] = fmaf(c1, acc[q], fmaf(c0, xc, xc));   // previous iterate 0
      else out[o] = acc[q];
    }
  }
}

__global__ void k_fill_hash(float* __restrict__ x, size_t count, unsigned seed) {
  for (size_t i = static_cast<size_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < count;
       i += static_cast<size_t>(gridDim.x) * blockDim.x) {
    unsigned h = static_cast<unsigned>(i) * 0x9E3779B1u ^ seed;
    h ^= h >> 16;
    h *= 0x85EBCA6Bu;
    h ^= h >> 13;
    h *= 0xC2B2AE35u;
    h ^= h >> 16;
    x[i] = static_cast<float>(h) * (2.f / 4294967296.f) - 1.f;
  }
}

// coarse[V] = sum over fine 2V + a, a in {-1,0,1}^3, of w(a) fine[2V + a] (R = I^T).
__global__ void __launch_bounds__(256) k_restrict(const float* __restrict__ fine, int nf,
                                                  float* __restrict__ coarse) {
  const int nc = nf / 2;
  const size_t Nf = static_cast<size_t>(nf) * nf * nf;
  const size_t Nc = static_cast<size_t>(nc) * nc * nc;
  for (size_t V = static_cast<size_t>(blockIdx.x) * blockDim.x + threadIdx.x; V < Nc;
       V += static_cast<size_t>(gridDim.x) * blockDim.x) {
    const int X = static_cast<int>(V % nc), Y = static_cast<int>((V / nc) % nc),
              Z = static_cast<int>(V / (static_cast<size_t>(nc) * nc));
    const Nb nb = make_nb(2 * X, 2 * Y, 2 * Z, nf);
    float acc[kPlanes];
#pragma unroll
    for (int q = 0; q < kPlanes; ++q) acc[q] = 0.f;
#pragma unroll
    for (int d = 0; d < 27; ++d) {
      const int dx = d % 3 - 1, dy = (d / 3) % 3 - 1, dz = d / 9 - 1;
      const float w = (dx ? 0.5f : 1.f) * (dy ? 0.5f : 1.f) * (dz ? 0.5f : 1.f);
      const size_t o = static_cast<size_t>(nb.X[dx + 1] + nb.Y[dy + 1] + nb.Z[dz + 1]);
#pragma unroll
      for (int q = 0; q < kPlanes; ++q) acc[q] = fmaf(w, __ldg(fine + q * Nf + o), acc[q]);
    }
#pragma unroll
    for (int q = 0; q < kPlanes; ++q) coarse[q * Nc + V] = acc[q];
  }
}

// fine (+)= I coarse. One thread per coarse cell (X..X+1, Y..Y+1, Z..Z+1): its 8 corner
// values give the 8 fine vertices (2X+a, 2Y+b, 2Z+c), a,b,c in {0,1}, by trilinear
// weights (1 on an even fine coordinate, 1/2 to each neighbour on an odd one).
__global__ void __launch_bounds__(256) k_prolong(const float* __restrict__ coarse, int nf,
                                                 float* __restrict__ fine, int overwrite) {
  const int nc = nf / 2;
  const size_t Nf = static_cast<size_t>(nf) * nf * nf;
  const size_t Nc = static_cast<size_t>(nc) * nc * nc;
  for (size_t V = static_cast<size_t>(blockIdx.x) * blockDim.x + threadIdx.x; V < Nc;
       V += static_cast<size_t>(gridDim.x) * blockDim.x) {
    const int X = static_cast<int>(V % nc), Y = static_cast<int>((V / nc) % nc),
              Z = static_cast<int>(V / (static_cast<size_t>(nc) * nc));
    const int X1 = X + 1 == nc ? 0 : X + 1, Y1 = Y + 1 == nc ? 0 : Y + 1, Z1 = Z + 1 == nc ? 0 : Z + 1;
    size_t cidx[8];
#pragma unroll
    for (int k = 0; k < 8; ++k)
      cidx[k] = static_cast<size_t>((k & 1) ? X1 : X) +
                static_cast<size_t>(nc) * (((k >> 1) & 1 ? Y1 : Y) + static_cast<size_t>(nc) * ((k >> 2) ? Z1 : Z));
    size_t fidx[8];
#pragma unroll
    for (int k = 0; k < 8; ++k)
      fidx[k] = static_cast<size_t>(2 * X + (k & 1)) +
                static_cast<size_t>(nf) * ((2 * Y + ((k >> 1) & 1)) + static_cast<size_t>(nf) * (2 * Z + (k >> 2)));
#pragma unroll 1
    for (int q = 0; q < kPlanes; ++q) {
      const float* cq = coarse + q * Nc;
      float c[8];
#pragma unroll
      for (int k = 0; k < 8; ++k) c[k] = __ldg(cq + cidx[k]);
      // interpolate along x, then y, then z
      float ax[8];
#pragma unroll
      for (int k = 0; k < 8; k += 2) {
        ax[k] = c[k];
        ax[k + 1] = 0.5f * (c[k] + c[k + 1]);
      }
      float ay[8];
#pragma unroll
      for (int zc = 0; zc < 2; ++zc)
#pragma unroll
        for (int a = 0; a < 2; ++a) {
          const float lo = ax[4 * zc + a], hi = ax[4 * zc + 2 + a];
          ay[4 * zc + a] = lo;
          ay[4 * zc + 2 + a] = 0.5f * (lo + hi);
        }
      float* fq = fine + q * Nf;
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        const float val = (k >> 2) ? 0.5f * (ay[k & 3] + ay[4 + (k & 3)]) : ay[k];
        fq[fidx[k]] = overwrite ? val : fq[fidx[k]] + val;
      }
    }
  }
}

// Dense FP64 matrix of the coarsest stencil: A[3v+r][3w+c] = block (v, d)[r][c],
// w = v + d wrapped (nc >= 3, so the 27 neighbours are distinct).
__global__ void k_coarsest_dense(const float* __restrict__ st, int nc, bool cb,
                                 double* __restrict__ A) {
  const size_t Nc = static_cast<size_t>(nc) * nc * nc;
  const int m = 3 * static_cast<int>(Nc);
  for (size_t it = static_cast<size_t>(blockIdx.x) * blockDim.x + threadIdx.x; it < 27 * Nc;
       it += static_cast<size_t>(gridDim.x) * blockDim.x) {
    const int d = static_cast<int>(it / Nc);
    const size_t v = it - static_cast<size_t>(d) * Nc;
    const int x = static_cast<int>(v % nc), y = static_cast<int>((v / nc) % nc),
              z = static_cast<int>(v / (static_cast<size_t>(nc) * nc));
    const int dx = d % 3 - 1, dy = (d / 3) % 3 - 1, dz = d / 9 - 1;
    const size_t w = static_cast<size_t>((x + dx + nc) % nc) +
                     static_cast<size_t>(nc) * (((y + dy + nc) % nc) + static_cast<size_t>(nc) * ((z + dz + nc) % nc));
    const size_t p = stencil_pos(x, y, z, nc, cb);
    for (int r = 0; r < 3; ++r)
      for (int c = 0; c < 3; ++c)
        A[(3 * v + r) * m + 3 * w + c] = static_cast<double>(st[static_cast<size_t>(9 * d + 3 * r + c) * Nc + p]);
  }
}

// In-place Gauss-Jordan inverse of the SPD block A[3:, 3:] (vertex 0 pinned, Sec. 4.2
// "eight corner vertices ... fixed"), no pivoting (SPD pivots are positive). One CTA.
// Row and column 0..2 are zeroed, giving the pinned inverse embedded in m x m.
__global__ void __launch_bounds__(1024) k_coarsest_invert(double* __restrict__ A, int m,
                                                          int* __restrict__ status) {
  __shared__ double piv_row[1536];
  __shared__ double piv_col[1536];
  for (int k = 3; k < m; ++k) {
    const double piv = A[static_cast<size_t>(k) * m + k];
    if (!(piv > 0.0)) {
      if (threadIdx.x == 0) *status = 1;
      return;
    }
    const double ip = 1.0 / piv;
    for (int j = threadIdx.x; j < m; j += blockDim.x) {
      piv_row[j] = A[static_cast<size_t>(k) * m + j];
      piv_col[j] = A[static_cast<size_t>(j) * m + k];
    }
    __syncthreads();
    for (size_t e = threadIdx.x; e < static_cast<size_t>(m) * m; e += blockDim.x) {
      const int i = static_cast<int>(e / m), j = static_cast<int>(e % m);
      if (i < 3 || j < 3) continue;
      double val;
      if (i == k && j == k) val = ip;
      else if (i == k) val = piv_row[j] * ip;
      else if (j == k) val = -piv_col[i] * ip;
      else val = A[e] - piv_col[i] * piv_row[j] * ip;
      A[e] = val;
    }
    __syncthreads();
  }
  for (size_t e = threadIdx.x; e < static_cast<size_t>(m) * m; e += blockDim.x) {
    const int i = static_cast<int>(e / m), j = static_cast<int>(e % m);
    if (i < 3 || j < 3) A[e] = 0.0;
  }
}

// G = P X P with P the projector removing the 3 rigid translations (per-component means):
// the centred pseudo-inverse of the coarsest operator (Sec. 4.2 null-space removal).
__global__ void __launch_bounds__(1024) k_coarsest_centre(const double* __restrict__ X, int m,
                                                          double* __restrict__ G) {
  extern __shared__ double sh[];          // rowmean[m*3] + tot[9]
  double* rmean = sh;                     // rmean[i*3 + b] = mean_w X[i][3w+b]
  double* tot = sh + 3 * m;
  const int nv = m / 3;
  for (int i = threadIdx.x; i < m; i += blockDim.x)
    for (int b = 0; b < 3; ++b) {
      double s = 0.0;
      for (int w = 0; w < nv; ++w) s += X[static_cast<size_t>(i) * m + 3 * w + b];
      rmean[i * 3 + b] = s / nv;
    }
  __syncthreads();
  if (threadIdx.x < 9) {
    const int a = threadIdx.x / 3, b = threadIdx.x % 3;
    double s = 0.0;
    for (int v = 0; v < nv; ++v) s += rmean[(3 * v + a) * 3 + b];
    tot[threadIdx.x] = s / nv;
  }
  __syncthreads();
  for (size_t e = threadIdx.x; e < static_cast<size_t>(m) * m; e += blockDim.x) {
    const int i = static_cast<int>(e / m), j = static_cast<int>(e % m);
    const int a = i % 3, b = j % 3;
    // X symmetric: column mean of column j over rows of component a = rmean[j][a]
    G[e] = X[e] - rmean[i * 3 + b] - rmean[j * 3 + a] + tot[a * 3 + b];
  }
}

// x = G b for the 6 cases (FP64 dot products), one warp per output row.
__global__ void __launch_bounds__(256) k_coarsest_apply(const double* __restrict__ G, int m,
                                                        const float* __restrict__ b,
                                                        float* __restrict__ x) {
  const int nv = m / 3;
  const int lane = threadIdx.x & 31;
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nwarps = (gridDim.x * blockDim.x) >> 5;
  for (int row = warp; row < kCases * m; row += nwarps) {
    const int c = row / m, i = row % m;
    double s = 0.0;
    for (int j = lane; j < m; j += 32) {
      const int w = j / 3, k = j % 3;
      s += G[static_cast<size_t>(i) * m + j] * static_cast<double>(b[static_cast<size_t>(3 * c + k) * nv + w]);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if (lane == 0) x[static_cast<size_t>(3 * c + i % 3) * nv + i / 3] = static_cast<float>(s);
  }
}

// Export a stencil in vertex-major order out[(v*27 + d)*9 + q].
__global__ void k_stencil_export(const float* __restrict__ st, int n, bool cb,
                                 float* __restrict__ out) {
  const size_t N = static_cast<size_t>(n) * n * n;
  for (size_t it = static_cast<size_t>(blockIdx.x) * blockDim.x + threadIdx.x; it < N * kStencil;
       it += static_cast<size_t>(gridDim.x) * blockDim.x) {
    const size_t v = it / kStencil;
    const int k = static_cast<int>(it % kStencil);
    const int x = static_cast<int>(v % n), y = static_cast<int>((v / n) % n),
              z = static_cast<int>(v / (static_cast<size_t>(n) * n));
    out[it] = st[static_cast<size_t>(k) * N + stencil_pos(x, y, z, n, cb)];
  }
}

}  // namespace

cudaError_t launch_level1_assemble(const homo_ctx* c, const Level& L1) {
  // the 18 KB table travels in the kernel's parameter bank (limit 32 KB)
  BfParam B;
  for (int i = 0; i < 8 * 576; ++i) B.b[i] = c->hBf[i];
  k_level1<<<grid_for(L1.N, 128), 128, 0, c->stream>>>(B, c->E, c->n, L1.st, L1.n, L1.colour_blocked);
  return cudaGetLastError();
}

cudaError_t launch_galerkin(const Level& Lf, const Level& Lc, float* tmp1, float* tmp2, cudaStream_t s) {
  const int n = Lf.n, h = n / 2;
  if (Lc.n != h || !Lf.colour_blocked) return cudaErrorInvalidValue;
  const size_t n1 = static_cast<size_t>(h) * n * n, n2 = static_cast<size_t>(h) * h * n;
  // x: level stencil -> (h, n, n) in tmp1; y: -> (h, h, n) in tmp2; z: -> the coarse level
  k_galerkin_axis<0><<<grid_for(27 * n1, 256), 256, 0, s>>>(Lf.st, n, n, n, true, tmp1, false);
  k_galerkin_axis<1><<<grid_for(27 * n2, 256), 256, 0, s>>>(tmp1, h, n, n, false, tmp2, false);
  k_galerkin_axis<2><<<grid_for(27 * Lc.N, 256), 256, 0, s>>>(tmp2, h, h, n, false, Lc.st, Lc.colour_blocked);
  return cudaGetLastError();
}

cudaError_t launch_coarse_residual(const Level& L, const float* b, const float* x, float* out,
                                   cudaStream_t s) {
  if (L.sth) k_coarse_residual<<<grid_for(L.N, 256), 256, 0, s>>>(L.sth, b, x, out, L.n, L.colour_blocked);
  else k_coarse_residual<<<grid_for(L.N, 256), 256, 0, s>>>(L.st, b, x, out, L.n, L.colour_blocked);
  return cudaGetLastError();
}

cudaError_t launch_coarse_gs(const Level& L, int colour, const float* f, float* x, int first,
                             cudaStream_t s) {
  const size_t h = static_cast<size_t>(L.n / 2);
  if (L.sth) k_coarse_gs<<<grid_for(h * h * h, 256), 256, 0, s>>>(L.sth, f, x, L.n, colour, first);
  else k_coarse_gs<<<grid_for(h * h * h, 256), 256, 0, s>>>(L.st, f, x, L.n, colour, first);
  return cudaGetLastError();
}

namespace {

template <typename T>
int cluster_fits(int size) {
  const void* fn = reinterpret_cast<const void*>(k_coarse_gs_cluster<T>);
  if (cudaFuncSetAttribute(fn, cudaFuncAttributeNonPortableClusterSizeAllowed, size > 8 ? 1 : 0) != cudaSuccess)
    return 0;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(size);
  cfg.blockDim = dim3(kClusterBlock);
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = size;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  int count = 0;
  if (cudaOccupancyMaxActiveClusters(&count, fn, &cfg) != cudaSuccess) return 0;
  return count;
}

std::mutex g_cluster_mu;
int g_cluster_size[256] = {};    // per device: 0 = not queried, -1 = no cluster launch
int g_resident_size[256] = {};   // per device: largest resident-form cluster, -1 = none
constexpr int kResidentSmemMax = 200 * 1024;   // dynamic; the static row scratch comes on top

int resident_fits(int size) {
  const void* fn = reinterpret_cast<const void*>(k_coarse_gs_resident);
  if (cudaFuncSetAttribute(fn, cudaFuncAttributeNonPortableClusterSizeAllowed, size > 8 ? 1 : 0) != cudaSuccess ||
      cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, kResidentSmemMax) != cudaSuccess)
    return 0;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(size);
  cfg.blockDim = dim3(kResThreads);
  cfg.dynamicSmemBytes = kResidentSmemMax;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = size;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  int count = 0;
  if (cudaOccupancyMaxActiveClusters(&count, fn, &cfg) != cudaSuccess) return 0;
  return count;
}

// Cluster size and per-CTA vertex count of the resident form on level L, or false when
// the level does not qualify (BF16 stencil, too many vertices, too much shared memory).
bool resident_shape(const Level& L, int cluster_max, int& csize, int& Mper, size_t& smem) {
  if (L.sth || cluster_max < 1 || L.n % 2) return false;
  const size_t h = static_cast<size_t>(L.n / 2), Nh = h * h * h;
  const size_t need = (Nh + kResVerts - 1) / kResVerts;
  int size = 1;
  while (size < cluster_max && static_cast<size_t>(size) < need) size *= 2;
  if (static_cast<size_t>(size) < need) return false;
  csize = size;
  Mper = static_cast<int>((Nh + size - 1) / size);
  smem = resident_smem_floats(L.N, Mper) * sizeof(float);
  return smem <= static_cast<size_t>(kResidentSmemMax);
}

}  // namespace

int coarse_cluster_size() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 256) {
    cudaGetLastError();
    return -1;
  }
  std::lock_guard<std::mutex> lk(g_cluster_mu);
  if (g_cluster_size[dev] == 0) {
    int best = -1;
    for (int size : {16, 8, 4}) {
      if (cluster_fits<float>(size) > 0 && cluster_fits<__nv_bfloat16>(size) > 0) {
        best = size;
        break;
      }
    }
    int res = -1;
    for (int size : {16, 8, 4, 2, 1}) {
      if (resident_fits(size) > 0) {
        res = size;
        break;
      }
    }
    cudaGetLastError();   // a refused size leaves its error behind
    g_cluster_size[dev] = best;
    g_resident_size[dev] = res;
  }
  return g_cluster_size[dev];
}

int coarse_resident_size() {
  coarse_cluster_size();   // runs the per-device queries once
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 256) {
    cudaGetLastError();
    return -1;
  }
  std::lock_guard<std::mutex> lk(g_cluster_mu);
  return g_resident_size[dev] == 0 ? -1 : g_resident_size[dev];
}

bool coarse_resident_ok(const Level& L, int cluster_max) {
  int csize, Mper;
  size_t smem;
  return resident_shape(L, cluster_max, csize, Mper, smem);
}

cudaError_t launch_coarse_gs_resident(const Level& L, int sweeps, int reverse, int first, const float* f,
                                      float* x, int cluster_max, cudaStream_t s) {
  int csize, Mper;
  size_t smem;
  if (!resident_shape(L, cluster_max, csize, Mper, smem)) return cudaErrorInvalidValue;
  const size_t h = static_cast<size_t>(L.n / 2), Nh = h * h * h;
  const int vec16 = (L.N % 4 == 0) && (Nh % 4 == 0) && (Mper % 4 == 0) &&
                    (reinterpret_cast<uintptr_t>(L.st) % 16 == 0);
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(kCases * csize);
  cfg.blockDim = dim3(kResThreads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = csize;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k_coarse_gs_resident, L.st, f, x, L.n, sweeps, reverse, first, csize, Mper,
                            vec16);
}

cudaError_t launch_coarse_gs_sweeps(const Level& L, int sweeps, int reverse, int first, const float* f,
                                    float* x, int cluster_max, cudaStream_t s) {
  const unsigned h = static_cast<unsigned>(L.n / 2);
  const size_t Nh = static_cast<size_t>(h) * h * h;
  // per case: the smallest power-of-two cluster with a thread per vertex of a colour, at
  // most cluster_max CTAs
  const size_t need = (Nh + kClusterBlock - 1) / kClusterBlock;
  int size = 1;
  while (size < cluster_max && static_cast<size_t>(size) < need) size *= 2;
  if (size > cluster_max) size = cluster_max;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(kCases * size);
  cfg.blockDim = dim3(kClusterBlock);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = size;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  if (L.sth)
    return cudaLaunchKernelEx(&cfg, k_coarse_gs_cluster<__nv_bfloat16>, L.sth, f, x, L.n, sweeps, reverse, first, size);
  return cudaLaunchKernelEx(&cfg, k_coarse_gs_cluster<float>, L.st, f, x, L.n, sweeps, reverse, first, size);
}

cudaError_t launch_coarse_gs_item(const Level& L, int colour, const float* f, float* x, int first,
                                  cudaStream_t s) {
  const unsigned h = static_cast<unsigned>(L.n / 2);
  const int g = grid_for(gs_items(h * h * h), kItemBlock);
  if (L.sth) k_coarse_gs_item<<<g, kItemBlock, 0, s>>>(L.sth, f, x, L.n, colour, first);
  else k_coarse_gs_item<<<g, kItemBlock, 0, s>>>(L.st, f, x, L.n, colour, first);
  return cudaGetLastError();
}

cudaError_t launch_coarse_cheb(const Level& L, const float* b, const float* x_in, float* out, int mode,
                               float c0, float c1, cudaStream_t s) {
  if (L.sth) k_coarse_cheb<<<grid_for(L.N, 256), 256, 0, s>>>(L.sth, b, x_in, out, L.n, L.colour_blocked, mode, c0, c1);
  else k_coarse_cheb<<<grid_for(L.N, 256), 256, 0, s>>>(L.st, b, x_in, out, L.n, L.colour_blocked, mode, c0, c1);
  return cudaGetLastError();
}

cudaError_t launch_coarse_dinvk(const Level& L, const float* x, float* y, cudaStream_t s) {
  if (L.sth) k_coarse_cheb<<<grid_for(L.N, 256), 256, 0, s>>>(L.sth, nullptr, x, y, L.n, L.colour_blocked, 2, 0.f, 0.f);
  else k_coarse_cheb<<<grid_for(L.N, 256), 256, 0, s>>>(L.st, nullptr, x, y, L.n, L.colour_blocked, 2, 0.f, 0.f);
  return cudaGetLastError();
}

cudaError_t launch_fill_hash(float* x, size_t count, unsigned seed, cudaStream_t s) {
  k_fill_hash<<<grid_for(count, 256), 256, 0, s>>>(x, count, seed);
  return cudaGetLastError();
}

cudaError_t launch_restrict(int nf, const float* fine, float* coarse, cudaStream_t s) {
  const size_t nc = static_cast<size_t>(nf / 2);
  k_restrict<<<grid_for(nc * nc * nc, 256), 256, 0, s>>>(fine, nf, coarse);
  return cudaGetLastError();
}

cudaError_t launch_prolong_add(int nf, const float* coarse, float* fine, int overwrite,
                               cudaStream_t s) {
  const size_t Nf = static_cast<size_t>(nf) * nf * nf;
  k_prolong<<<grid_for(Nf / 8, 256), 256, 0, s>>>(coarse, nf, fine, overwrite);
  return cudaGetLastError();
}

cudaError_t launch_coarsest_setup(homo_ctx* c) {
  const Level& L = c->lev[c->nlev - 1];
  const int m = c->mc;
  cudaError_t e = cudaMemsetAsync(c->A, 0, sizeof(double) * m * m, c->stream);
  if (e != cudaSuccess) return e;
  k_coarsest_dense<<<grid_for(27 * L.N, 256), 256, 0, c->stream>>>(L.st, L.n, L.colour_blocked, c->A);
  int* status = reinterpret_cast<int*>(c->scal + S_OC + 63);
  e = cudaMemsetAsync(status, 0, sizeof(int), c->stream);
  if (e != cudaSuccess) return e;
  k_coarsest_invert<<<1, 1024, 0, c->stream>>>(c->A, m, status);
  const size_t shm = sizeof(double) * (3 * m + 9);
  e = cudaFuncSetAttribute(k_coarsest_centre, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           static_cast<int>(shm));
  if (e != cudaSuccess) return e;
  k_coarsest_centre<<<1, 1024, shm, c->stream>>>(c->A, m, c->G);
  return cudaGetLastError();
}

cudaError_t launch_coarsest_apply(const homo_ctx* c, const float* b, float* x) {
  const int rows = kCases * c->mc;
  const int blocks = (rows * 32 + 255) / 256;
  k_coarsest_apply<<<blocks < 1216 ? blocks : 1216, 256, 0, c->stream>>>(c->G, c->mc, b, x);
  return cudaGetLastError();
}

cudaError_t launch_stencil_bf16(const Level& L, cudaStream_t s) {
  if (!L.sth || !L.st) return cudaErrorInvalidValue;
  k_stencil_bf16<<<grid_for(27 * L.N, 256), 256, 0, s>>>(L.st, L.n, L.colour_blocked, L.sth);
  return cudaGetLastError();
}

cudaError_t launch_stencil_export(const Level& L, float* out, cudaStream_t s) {
  k_stencil_export<<<grid_for(L.N * kStencil, 256), 256, 0, s>>>(L.st, L.n, L.colour_blocked, out);
  return cudaGetLastError();
}

}  // namespace homo
