// Finest-level kernels. The level-0 stiffness is never stored (Sec. 4.1): every kernel
// rebuilds what it needs from the element moduli E and the element matrix K0, which sits
// in the kernel's parameter (constant) bank.
//
// Vertex form of K u (Eq. 13): incident element t = a + 2b + 4c of vertex v has origin
// v - (1,1,1) + (a,b,c) and v is its local vertex 7 - t. The 3x3 coupling block between v
// and its neighbour v + d is
//     A_d = sum over (t, j) with bits(t) + bits(j) - 1 = d of E_t * K0[7 - t, j],
// built once per vertex and applied to all 6 load cases (the 6 cases share E and K0).
#include <mutex>
#include <string>

#include "dev_common.cuh"
#include "stencil.cuh"

namespace homo {

namespace {

// Error-free transformations (Knuth TwoSum, FMA-based TwoProduct) with operations the
// compiler may not contract or reorder.
__device__ __forceinline__ f32x2 fmul2(f32x2 a, f32x2 b) {
  f32x2 d;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}

__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bb = __fadd_rn(s, -a);
  e = __fadd_rn(__fadd_rn(a, -__fadd_rn(s, -bb)), __fadd_rn(b, -bb));
}

// Macro-strain loads in vertex form (Eq. 11): f_(i,v) = sum_t E_t (K0 chi_i)[7 - t].
// In a uniform medium the 8 element forces at a vertex cancel exactly (sum_t (K0
// chi_i)[7 - t] = 0), so the kernel sums (E_t - E_0) (K0 chi_i)[7 - t]: the loads are
// exactly zero where E is locally uniform and carry no cancellation error elsewhere.
// The sum is formed in double-float arithmetic (the difference E_t - E_0 and K0 chi split
// exactly, error-free products and sums) and stored as f + flo: an FP32 load rounded
// against the largest of its terms perturbs the weakly held soft-region displacements,
// whose strain energies the sensitivities of Eq. 9 weigh.
__global__ void __launch_bounds__(256) k_loads(const __grid_constant__ LoadParam L,
                                               const float* __restrict__ E,
                                               float* __restrict__ f, float* __restrict__ flo, int n) {
  const size_t N = static_cast<size_t>(n) * n * n;
  for (size_t v = static_cast<size_t>(blockIdx.x) * blockDim.x + threadIdx.x; v < N;
       v += static_cast<size_t>(gridDim.x) * blockDim.x) {
    int x, y, z;
    decode3(static_cast<unsigned>(v), static_cast<unsigned>(n), x, y, z);
    const Nb nb = make_nb(x, y, z, n);
    float Et[8];
    load_E8(E, nb, Et);
    float dh[8], dl[8];
#pragma unroll
    for (int t = 1; t < 8; ++t) two_sum(Et[t], -Et[0], dh[t], dl[t]);   // E_t - E_0 = dh + dl
#pragma unroll
    for (int c = 0; c < kCases; ++c)
#pragma unroll
      for (int r = 0; r < 3; ++r) {
        float hi = 0.f, lo = 0.f;
#pragma unroll
        for (int t = 1; t < 8; ++t) {
          const float a = L.fe[c][3 * (7 - t) + r], al = L.fe_lo[c][3 * (7 - t) + r];
          const float p = __fmul_rn(dh[t], a);
          const float pe = fmaf(dh[t], a, -p);               // dh a = p + pe exactly
          float s, e;
          two_sum(hi, p, s, e);
          hi = s;
          lo = __fadd_rn(lo, __fadd_rn(__fadd_rn(e, pe), fmaf(dh[t], al, __fmul_rn(dl[t], a))));
        }
        const float s2 = __fadd_rn(hi, lo);
        const size_t o = static_cast<size_t>(3 * c + r) * N + v;
        f[o] = s2;
        flo[o] = __fadd_rn(lo, -__fadd_rn(s2, -hi));          // FastTwoSum: f + flo = hi + lo
      }
  }
}


// r = (b + blo) - K (u + ulo) evaluated in double-float arithmetic (difference form, products
// and sums error-free up to the final rounding), then partials of ||r_c||^2 and of the
// 18 plane sums. This is the accurate true residual the CG driver restarts from; it uses
// exactly the FP32 blocks A_d of the CG product, so both see the same operator.
__global__ void __launch_bounds__(128) k_fine_true_residual(const __grid_constant__ KeParam K,
                                                            const float* __restrict__ E,
                                                            const float* __restrict__ u,
                                                            const float* __restrict__ ulo,
                                                            const float* __restrict__ b,
                                                            const float* __restrict__ blo,
                                                            float* __restrict__ out, int n,
                                                            double* __restrict__ part) {
  const size_t N = static_cast<size_t>(n) * n * n;
  float red[kCases + kPlanes];
#pragma unroll
  for (int c = 0; c < kCases + kPlanes; ++c) red[c] = 0.f;
  for (size_t v = static_cast<size_t>(blockIdx.x) * blockDim.x + threadIdx.x; v < N;
       v += static_cast<size_t>(gridDim.x) * blockDim.x) {
    int x, y, z;
    decode3(static_cast<unsigned>(v), static_cast<unsigned>(n), x, y, z);
    const Nb nb = make_nb(x, y, z, n);
    float Et[8];
    load_E8(E, nb, Et);
    // The 6 cases advance in pairs (2p, 2p + 1) on the two lanes of f32x2 registers. Every
    // lane performs exactly the scalar operations of the double-float recurrence below,
    // in the same order (the negated-operand forms are exact: round to nearest is
    // symmetric), so the result is bitwise that of a scalar evaluation:
    //   dh + e = u_(v+d) - u_v (two-sum), dl = e + (ulo_(v+d) - ulo_v),
    //   p = a dh, pe = a dh - p (FMA), hi + e' = hi + p (two-sum),
    //   lo += e' + (a dl + pe).
    f32x2 hi[9], lo[9], nown[9], ownlo[9];
#pragma unroll
    for (int p = 0; p < 3; ++p)
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        const int q0 = 6 * p + k, q1 = q0 + 3;
        hi[3 * p + k] = 0ull;
        lo[3 * p + k] = 0ull;
        nown[3 * p + k] = pack2(-__ldg(u + q0 * N + v), -__ldg(u + q1 * N + v));
        ownlo[3 * p + k] = pack2(__ldg(ulo + q0 * N + v), __ldg(ulo + q1 * N + v));
      }
#pragma unroll 1
    for (int d = 0; d < 27; ++d) {
      if (d == 13) continue;
      const int dx = d % 3 - 1, dy = (d / 3) % 3 - 1, dz = d / 9 - 1;
      float A[9];
      // runtime d: the block is rebuilt with runtime offsets (same FP32 operations and
      // order as the compile-time version in the CG product)
      nb_block(K, Et, dx, dy, dz, A);
      f32x2 Ap[9], An[9];
#pragma unroll
      for (int e = 0; e < 9; ++e) {
        Ap[e] = pack2(A[e], A[e]);
        An[e] = pack2(-A[e], -A[e]);
      }
      const size_t w = static_cast<size_t>(nb.X[dx + 1] + nb.Y[dy + 1] + nb.Z[dz + 1]);
#pragma unroll
      for (int p = 0; p < 3; ++p) {
        f32x2 dh[3], dl[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
          const size_t o0 = static_cast<size_t>(6 * p + k) * N + w, o1 = o0 + 3 * N;
          const f32x2 a = pack2(__ldg(u + o0), __ldg(u + o1));
          const f32x2 b = nown[3 * p + k];
          const f32x2 s = fadd2(a, b);                      // two-sum of u_(v+d) and -u_v
          const f32x2 bb = fsub2(s, a);
          const f32x2 e = fadd2(fsub2(a, fsub2(s, bb)), fsub2(b, bb));
          dh[k] = s;
          dl[k] = fadd2(e, fsub2(pack2(__ldg(ulo + o0), __ldg(ulo + o1)), ownlo[3 * p + k]));
        }
#pragma unroll
        for (int r = 0; r < 3; ++r)
#pragma unroll
          for (int k = 0; k < 3; ++k) {
            const f32x2 pr = fmul2(Ap[3 * r + k], dh[k]);
            const f32x2 npe = ffma2(An[3 * r + k], dh[k], pr);      // = -(a dh - p) exactly
            const f32x2 h = hi[3 * p + r];
            const f32x2 s = fadd2(h, pr);                            // two-sum of hi and p
            const f32x2 bb = fsub2(s, h);
            const f32x2 e = fadd2(fsub2(h, fsub2(s, bb)), fsub2(pr, bb));
            hi[3 * p + r] = s;
            // e + (a dl + pe) = e - (-a dl - pe) = e - fma(-a, dl, -pe)
            lo[3 * p + r] = fadd2(lo[3 * p + r], fsub2(e, ffma2(An[3 * r + k], dl[k], npe)));
          }
      }
    }
    float hs[kPlanes], ls[kPlanes];
#pragma unroll
    for (int p = 0; p < 3; ++p)
#pragma unroll
      for (int r = 0; r < 3; ++r) {
        unpack2(hi[3 * p + r], hs[6 * p + r], hs[6 * p + 3 + r]);
        unpack2(lo[3 * p + r], ls[6 * p + r], ls[6 * p + 3 + r]);
      }
#pragma unroll
    for (int q = 0; q < kPlanes; ++q) {
      const size_t o = static_cast<size_t>(q) * N + v;
      float s, e;
      two_sum(__ldg(b + o), -hs[q], s, e);
      const float val = __fadd_rn(s, __fadd_rn(e, __fadd_rn(__ldg(blo + o), -ls[q])));
      out[o] = val;
      red[q / 3] = fmaf(val, val, red[q / 3]);
      red[kCases + q] += val;
    }
  }
  block_sum_store<kCases + kPlanes>(red, part);
}

// First Chebyshev step from x = 0: out_v = c0 S_v^-1 (b_v - bmean), S_v the diagonal
// block (the Gauss-Seidel diagonal solve of Eq. 16).
__global__ void __launch_bounds__(256) k_fine_jacobi_start(const __grid_constant__ KeParam K,
                                                           const float* __restrict__ E,
                                                           const float* __restrict__ b,
                                                           const double* __restrict__ bmean,
                                                           float* __restrict__ out, int n, float c0) {
  const size_t N = static_cast<size_t>(n) * n * n;
  for (size_t v = static_cast<size_t>(blockIdx.x) * blockDim.x + threadIdx.x; v < N;
       v += static_cast<size_t>(gridDim.x) * blockDim.x) {
    const int x = static_cast<int>(v % n), y = static_cast<int>((v / n) % n),
              z = static_cast<int>(v / (static_cast<size_t>(n) * n));
    const Nb nb = make_nb(x, y, z, n);
    float Et[8];
    load_E8(E, nb, Et);
    float S[9];
    nb_block(K, Et, 0, 0, 0, S);
    float rhs[kPlanes];
#pragma unroll
    for (int q = 0; q < kPlanes; ++q)
      rhs[q] = __ldg(b + q * N + v) - (bmean ? static_cast<float>(bmean[q]) : 0.f);
    solve3x6(S, rhs);
#pragma unroll
    for (int q = 0; q < kPlanes; ++q) out[q * N + v] = c0 * rhs[q];
  }
}

// Level-0 stencil written out (used only when the finest level is also the coarsest and
// is solved directly): st[(9d + q) * N + pos(v)] = A_d[q].
__global__ void __launch_bounds__(256) k_fine_stencil(const __grid_constant__ KeParam K,
                                                      const float* __restrict__ E, int n, bool cb,
                                                      float* __restrict__ st) {
  const size_t N = static_cast<size_t>(n) * n * n;
  for (size_t v = static_cast<size_t>(blockIdx.x) * blockDim.x + threadIdx.x; v < N;
       v += static_cast<size_t>(gridDim.x) * blockDim.x) {
    const int x = static_cast<int>(v % n), y = static_cast<int>((v / n) % n),
              z = static_cast<int>(v / (static_cast<size_t>(n) * n));
    const Nb nb = make_nb(x, y, z, n);
    float Et[8];
    load_E8(E, nb, Et);
    const size_t p = stencil_pos(x, y, z, n, cb);
#pragma unroll
    for (int d = 0; d < 27; ++d) {
      float A[9];
      nb_block(K, Et, d % 3 - 1, (d / 3) % 3 - 1, d / 9 - 1, A);
#pragma unroll
      for (int q = 0; q < 9; ++q) st[static_cast<size_t>(9 * d + q) * N + p] = A[q];
    }
  }
}

__global__ void k_simp(const float* __restrict__ rin, float* __restrict__ rout,
                       float* __restrict__ E, size_t N, float p, float E0, float Emin) {
  for (size_t e = static_cast<size_t>(blockIdx.x) * blockDim.x + threadIdx.x; e < N;
       e += static_cast<size_t>(gridDim.x) * blockDim.x) {
    float r = rin[e];
    r = fminf(fmaxf(r, 0.f), 1.f);
    rout[e] = r;
    E[e] = Emin + powf(r, p) * (E0 - Emin);
  }
}

struct ElemParam {
  float mu[kCases];           // eigenvalues of the symmetrised objective gradient G
  float vec[kCases][kCases];  // vec[k][i]: component i of the eigenvector of mu[k]
  float p, dE;                // SIMP exponent, E0 - Emin
  float invN;
};

constexpr int kElemCases = kCases;            // one warp per load case
constexpr int kElemBlock = 32 * kElemCases;   // 32 elements x 6 cases
constexpr int kElemPad = 25;                  // w row stride in shared memory (bank spread)

// Pair slot of (i, j) in the row-major upper triangle of the 6x6 C^H (i <= j).
__host__ __device__ constexpr int pair_slot(int i, int j) {
  return i <= j ? i * kCases - i * (i - 1) / 2 + (j - i) : j * kCases - j * (j - 1) / 2 + (i - j);
}

// Per element q_ij = w_i^T K0 w_j, w_i = chi_i - (u_i - u_i at local vertex 0): the
// summand of Eq. 7 (subtracting the element's own translation leaves K0 w unchanged and
// keeps FP32 round-off independent of the field's magnitude, cf. Sec. 4.2 "relative
// coordinate"). Six threads per element, one per load case i and each in its own warp,
// so a warp's loads cover 32 consecutive elements: thread i gathers w_i (both parts of
// the double-float field), forms y_i = K0 w_i and the products q_ij = y_i . w_j of the
// pairs dealt to it (q_ij = q_ji: the diagonal, i+1, i+2 and, for i < 3, i+3 mod 6, so
// 3 or 4 each), reading the other w_j from shared memory.
// MODE 0: block partial sums of E_e q_ij (21 values, Kahan-compensated per thread).
// MODE 1: sensitivity (Eq. 8-9) p rho^(p-1) dE sum_ij g_ij q_ij / N, evaluated as
// sum_k mu_k z_k^T K0 z_k with G = sym(g) = sum_k mu_k v_k v_k^T and z_k = sum_i v_k[i] w_i
// (thread k forms z_k from the six w_i in shared memory): each term is a non-negative
// quadratic form, so the sum does not cancel across the 21 products (for the bulk
// objective G has rank one and the sensitivity is a single quadratic form).
template <int MODE>
__global__ void __launch_bounds__(kElemBlock) k_fine_elem(const __grid_constant__ KeParam K,
                                                          const __grid_constant__ ChiParam X,
                                                          const __grid_constant__ ElemParam P,
                                                          const float* __restrict__ E,
                                                          const float* __restrict__ rho,
                                                          const float* __restrict__ u,
                                                          const float* __restrict__ ulo, int n,
                                                          float* __restrict__ sens,
                                                          double* __restrict__ part) {
  __shared__ float ws[kElemCases][32][kElemPad];
  __shared__ float sp[kElemCases][32];
  __shared__ double sacc[21];
  const int lane = threadIdx.x & 31, i = threadIdx.x >> 5;   // element slot, load case
  const size_t N = static_cast<size_t>(n) * n * n;
  const int npair = i < 3 ? 4 : 3;
  int jp[4], slot[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    jp[k] = (i + k) % kCases;
    slot[k] = pair_slot(i, jp[k]);
  }
  float cs[4] = {0.f, 0.f, 0.f, 0.f}, cc[4] = {0.f, 0.f, 0.f, 0.f};
  for (size_t e0 = static_cast<size_t>(blockIdx.x) * 32; e0 < N; e0 += static_cast<size_t>(gridDim.x) * 32) {
    const size_t e = e0 + lane;
    const bool live = e < N;
    float w[24];
    if (live) {
      int x, y, z;
      decode3(static_cast<unsigned>(e), static_cast<unsigned>(n), x, y, z);
      const int xs[2] = {x, x == n - 1 ? 0 : x + 1};
      const int ys[2] = {y * n, (y == n - 1 ? 0 : y + 1) * n};
      const int zs[2] = {z * n * n, (z == n - 1 ? 0 : z + 1) * n * n};
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        const float* uq = u + static_cast<size_t>(3 * i + k) * N;
        const float* lq = ulo + static_cast<size_t>(3 * i + k) * N;
        const float h0 = __ldg(uq + e), l0 = __ldg(lq + e);
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          const size_t vj = static_cast<size_t>(xs[j & 1] + ys[(j >> 1) & 1] + zs[j >> 2]);
          const float du = (__ldg(uq + vj) - h0) + (__ldg(lq + vj) - l0);
          w[3 * j + k] = X.chi[i][3 * j + k] - du;
        }
      }
    } else {
#pragma unroll
      for (int r = 0; r < 24; ++r) w[r] = 0.f;
    }
#pragma unroll
    for (int r = 0; r < 24; ++r) ws[i][lane][r] = w[r];
    __syncthreads();
    if (MODE == 1) {   // z_k = sum_i v_k[i] w_i replaces w: thread i now stands for mode k = i
#pragma unroll
      for (int r = 0; r < 24; ++r) {
        float zr = 0.f;
#pragma unroll
        for (int c = 0; c < kCases; ++c) zr = fmaf(P.vec[i][c], ws[c][lane][r], zr);
        w[r] = zr;
      }
    }
    float yv[24];
#pragma unroll
    for (int r = 0; r < 24; ++r) yv[r] = 0.f;
#pragma unroll
    for (int k = 0; k < 24; ++k) {
#pragma unroll
      for (int r = 0; r < 24; ++r) yv[r] = fmaf(K.k[r * 24 + k], w[k], yv[r]);
    }
    float q[4] = {0.f, 0.f, 0.f, 0.f};
    if (MODE == 1) {
      float t = 0.f;
#pragma unroll
      for (int r = 0; r < 24; ++r) t = fmaf(yv[r], w[r], t);
      q[0] = P.mu[i] * t;
    } else {
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        float sdot = 0.f;
        if (k < npair) {
          const float* wj = ws[jp[k]][lane];
#pragma unroll
          for (int r = 0; r < 24; ++r) sdot = fmaf(yv[r], wj[r], sdot);
        }
        q[k] = sdot;
      }
    }
    if (MODE == 0) {
      if (live) {
        const float Ee = __ldg(E + e);
#pragma unroll
        for (int k = 0; k < 4; ++k) {   // Kahan summation of E_e q_e,k
          const float yk = fmaf(Ee, q[k], -cc[k]);
          const float t = cs[k] + yk;
          cc[k] = (t - cs[k]) - yk;
          cs[k] = t;
        }
      }
    } else {
      sp[i][lane] = q[0];
    }
    __syncthreads();
    if (MODE == 1 && i == 0 && live) {
      float sg = 0.f;
#pragma unroll
      for (int c = 0; c < kElemCases; ++c) sg += sp[c][lane];
      const float r = __ldg(rho + e);
      sens[e] = P.p * powf(r, P.p - 1.f) * P.dE * sg * P.invN;
    }
  }
  if (MODE == 0) {
    // each pair slot belongs to exactly one warp: reduce the warp's 32 sums per slot
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      float v = cs[k];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
      if (lane == 0 && k < npair) sacc[slot[k]] = static_cast<double>(v);
    }
    __syncthreads();
    if (threadIdx.x < 21) part[static_cast<size_t>(blockIdx.x) * 21 + threadIdx.x] = sacc[threadIdx.x];
  }
}

}  // namespace

cudaError_t launch_simp(const float* rho_in, float* rho_out, float* E, size_t N, float p,
                        float E0, float Emin, cudaStream_t s) {
  k_simp<<<grid_for(N, 256), 256, 0, s>>>(rho_in, rho_out, E, N, p, E0, Emin);
  return cudaGetLastError();
}

cudaError_t launch_fine_jacobi_start(const homo_ctx* c, const float* b, const double* bmean, float* out,
                                     float c0) {
  k_fine_jacobi_start<<<grid_for(c->N, 256), 256, 0, c->stream>>>(c->ke, c->E, b, bmean, out, c->n, c0);
  return cudaGetLastError();
}

cudaError_t launch_fine_stencil(const homo_ctx* c, const Level& L0) {
  k_fine_stencil<<<grid_for(c->N, 256), 256, 0, c->stream>>>(c->ke, c->E, c->n, L0.colour_blocked, L0.st);
  return cudaGetLastError();
}

cudaError_t launch_loads(const homo_ctx* c, float* f) {
  k_loads<<<grid_for(c->N, 256), 256, 0, c->stream>>>(c->ld, c->E, f, c->flo, c->n);
  return cudaGetLastError();
}

cudaError_t launch_fine_apply(const homo_ctx* c, const float* u, float* out, double* part,
                              int* grid_out) {
  return launch_fine_tiled(c, 1, u, nullptr, out, part, grid_out);
}

cudaError_t launch_fine_residual(const homo_ctx* c, const float* b, const float* u,
                                 const float* ulo, float* out, double* part, int* grid_out,
                                 const double* bmean) {
  if (ulo) {
    const int g = grid_for(c->N, 128);
    if (grid_out) *grid_out = g;
    k_fine_true_residual<<<g, 128, 0, c->stream>>>(c->ke, c->E, u, ulo, b, c->flo, out, c->n, part);
    return cudaGetLastError();
  }
  return launch_fine_tiled(c, 3, u, b, out, nullptr, grid_out, bmean);
}


cudaError_t launch_fine_elem(const homo_ctx* c, int mode, const double* g36, float* sens,
                             double* part, int* grid_out) {
  ElemParam P{};
  if (g36) {   // sum_ij g_ij q_ij = sum_ij G_ij q_ij, G = (g + g^T) / 2 = sum_k mu_k v_k v_k^T
    double G[kCases * kCases], V[kCases * kCases];
    for (int i = 0; i < kCases; ++i)
      for (int j = 0; j < kCases; ++j) G[i * kCases + j] = 0.5 * (g36[6 * i + j] + g36[6 * j + i]);
    sym_eigen(kCases, G, V);
    for (int k = 0; k < kCases; ++k) {
      P.mu[k] = static_cast<float>(G[k * kCases + k]);
      for (int i = 0; i < kCases; ++i) P.vec[k][i] = static_cast<float>(V[i * kCases + k]);
    }
  }
  P.p = static_cast<float>(c->p);
  P.dE = static_cast<float>(c->E0 - c->Emin);
  P.invN = static_cast<float>(1.0 / static_cast<double>(c->N));
  const int g = grid_for((c->N + 31) / 32, 1);   // one block per 32 elements, capped
  if (grid_out) *grid_out = g;
  if (mode == 0)
    k_fine_elem<0><<<g, kElemBlock, 0, c->stream>>>(c->ke, c->chi, P, c->E, c->rho, c->u, c->ulo,
                                                   c->n, sens, part);
  else
    k_fine_elem<1><<<g, kElemBlock, 0, c->stream>>>(c->ke, c->chi, P, c->E, c->rho, c->u, c->ulo,
                                                   c->n, sens, part);
  return cudaGetLastError();
}

void set_thread_error(const std::string& msg);

// ---------------------------------------------------------------- allocation-free C^H
// A second way to evaluate C^H for callers that cannot allocate device memory while
// they run. Its per-block partial sums go to one fixed array in device memory that the
// library reserves when it is loaded, instead of to context buffers from cudaMalloc.
namespace {

constexpr int kNoAllocBlocks = 1216;   // partial-sum rows: 152 SMs x 8 blocks
constexpr int kNoAllocMaxN = 1024;     // largest cell per axis (indices stay in int)

// Rows 0..kNoAllocBlocks-1: 21 partial sums per block; last row: the 21 totals.
// Every GPU that loads the library holds this array (about 200 KB) until exit.
static __device__ __align__(256) double g_noalloc_scratch[(kNoAllocBlocks + 1) * 21];

std::mutex g_noalloc_mu;
double* g_noalloc_ptr[256] = {};   // device address of g_noalloc_scratch, per device

// Thread per element, its 144 w values and 21 products in a shared-memory row.
constexpr int kNoAllocElemBlock = 128;
constexpr int kNoAllocStride = 165;   // 144 w values + 21 products per thread row (odd: bank spread)

// The element arithmetic of Eq. 7 (w_i = chi_i - relative displacement, q_ij = w_i^T K0
// w_j, Kahan sums of E_e q_ij) with one thread per element; ulo may be null (read as 0).
__global__ void __launch_bounds__(kNoAllocElemBlock) k_ch_noalloc(const __grid_constant__ KeParam K,
                                                           const __grid_constant__ ChiParam X,
                                                           const float* __restrict__ E,
                                                           const float* __restrict__ u,
                                                           const float* __restrict__ ulo, int n,
                                                           double* __restrict__ scratch) {
  extern __shared__ float wsh[];
  float* w = wsh + threadIdx.x * kNoAllocStride;
  const size_t N = static_cast<size_t>(n) * n * n;
  float cs[21], cc[21];
#pragma unroll
  for (int k = 0; k < 21; ++k) cs[k] = cc[k] = 0.f;
  for (size_t e = static_cast<size_t>(blockIdx.x) * blockDim.x + threadIdx.x; e < N;
       e += static_cast<size_t>(gridDim.x) * blockDim.x) {
    const int x = static_cast<int>(e % n), y = static_cast<int>((e / n) % n),
              z = static_cast<int>(e / (static_cast<size_t>(n) * n));
    const int xs[2] = {x, x == n - 1 ? 0 : x + 1};
    const int ys[2] = {y * n, (y == n - 1 ? 0 : y + 1) * n};
    const int zs[2] = {z * n * n, (z == n - 1 ? 0 : z + 1) * n * n};
#pragma unroll
    for (int q = 0; q < kPlanes; ++q) {
      const float* uq = u + static_cast<size_t>(q) * N;
      const float* lq = ulo ? ulo + static_cast<size_t>(q) * N : nullptr;
      const float h0 = __ldg(uq + e), l0 = lq ? __ldg(lq + e) : 0.f;
      const int c = q / 3, k = q % 3;
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const size_t vj = static_cast<size_t>(xs[j & 1] + ys[(j >> 1) & 1] + zs[j >> 2]);
        const float du = (__ldg(uq + vj) - h0) + (lq ? (__ldg(lq + vj) - l0) : 0.f);
        w[c * 24 + 3 * j + k] = X.chi[c][3 * j + k] - du;
      }
    }
    float* q = w + 144;
#pragma unroll 1
    for (int i = 0, idx = 0; i < kCases; ++i) {
      float yv[24];
#pragma unroll
      for (int r = 0; r < 24; ++r) yv[r] = 0.f;
#pragma unroll
      for (int k = 0; k < 24; ++k) {
        const float wk = w[i * 24 + k];
#pragma unroll
        for (int r = 0; r < 24; ++r) yv[r] = fmaf(K.k[r * 24 + k], wk, yv[r]);
      }
#pragma unroll 1
      for (int j = i; j < kCases; ++j, ++idx) {
        float s = 0.f;
#pragma unroll
        for (int k = 0; k < 24; ++k) s = fmaf(yv[k], w[j * 24 + k], s);
        q[idx] = s;
      }
    }
    const float Ee = __ldg(E + e);
#pragma unroll
    for (int k = 0; k < 21; ++k) {
      const float yk = fmaf(Ee, q[k], -cc[k]);
      const float t = cs[k] + yk;
      cc[k] = (t - cs[k]) - yk;
      cs[k] = t;
    }
  }
  block_sum_store<21>(cs, scratch);
}

// totals[k] = sum over the nblk rows written by this call, fixed order.
__global__ void k_ch_noalloc_total(double* __restrict__ scratch, int nblk) {
  const int k = threadIdx.x;
  if (k >= 21) return;
  double s = 0.0;
  for (int b = 0; b < nblk; ++b) s += scratch[static_cast<size_t>(b) * 21 + k];
  scratch[static_cast<size_t>(kNoAllocBlocks) * 21 + k] = s;
}

int noalloc_fail(int code, const std::string& msg) {
  set_thread_error(msg);
  return code;
}

}  // namespace

}  // namespace homo

extern "C" int homo_CH_noalloc(int n, double nu, const float* E, const float* u, const float* ulo,
                               double CH[36], void* cuda_stream) {
  using namespace homo;
  if (n < 4 || n > kNoAllocMaxN)
    return noalloc_fail(HOMO_EINVAL, "homo_CH_noalloc: n = " + std::to_string(n) +
                                         " is outside [4, " + std::to_string(kNoAllocMaxN) +
                                         "], the largest cell its fixed scratch array serves");
  if (!(nu > -1.0 && nu < 0.5) || !E || !u || !CH)
    return noalloc_fail(HOMO_EINVAL, "homo_CH_noalloc: bad nu or null pointer");
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess || dev < 0 || dev >= 256)
    return noalloc_fail(HOMO_ECUDA, std::string("homo_CH_noalloc: cudaGetDevice: ") + cudaGetErrorString(e));
  double* scratch = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
      void* p = nullptr;
      e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
      if (e != cudaSuccess || !p)
        return noalloc_fail(HOMO_ECUDA, std::string("homo_CH_noalloc: cudaGetSymbolAddress: ") +
                                            cudaGetErrorString(e));
      g_noalloc_ptr[dev] = static_cast<double*>(p);
    }
    scratch = g_noalloc_ptr[dev];
  }
  KeParam ke;
  LoadParam ld;
  ChiParam chi;
  build_element_matrix(nu, ke, ld, chi);
  const size_t N = static_cast<size_t>(n) * n * n;
  size_t blocks = (N + kNoAllocElemBlock - 1) / kNoAllocElemBlock;
  if (blocks > static_cast<size_t>(kNoAllocBlocks)) blocks = kNoAllocBlocks;
  const size_t shm = static_cast<size_t>(kNoAllocElemBlock) * kNoAllocStride * sizeof(float);
  e = cudaFuncSetAttribute(k_ch_noalloc, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(shm));
  if (e == cudaSuccess) {
    k_ch_noalloc<<<static_cast<int>(blocks), kNoAllocElemBlock, shm, s>>>(ke, chi, E, u, ulo, n, scratch);
    k_ch_noalloc_total<<<1, 32, 0, s>>>(scratch, static_cast<int>(blocks));
    e = cudaGetLastError();
  }
  double tot[21];
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(tot, scratch + static_cast<size_t>(kNoAllocBlocks) * 21, sizeof(tot),
                        cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess)
    return noalloc_fail(HOMO_ECUDA, std::string("homo_CH_noalloc: ") + cudaGetErrorString(e));
  const double invN = 1.0 / static_cast<double>(N);
  int idx = 0;
  for (int i = 0; i < kCases; ++i)
    for (int j = i; j < kCases; ++j) {
      CH[6 * i + j] = CH[6 * j + i] = tot[idx++] * invN;
    }
  return HOMO_OK;
}
