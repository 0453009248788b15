// Tiled finest-level stencil kernels: each block owns a 32 x 8 column of vertices over a
// chunk of z planes and marches along z. Four planes of the 6-case field (with a
// one-vertex periodic halo) and three planes of element moduli live in shared memory;
// the plane two steps ahead is fetched with asynchronous copies (cp.async) while the
// current plane is computed, so global latency overlaps the arithmetic. Each thread
// builds the 27 coupling blocks A_d of its vertex (Eq. 13) from the moduli and the
// element matrix in the parameter bank and applies them to the 6 load cases.
#include "stencil.cuh"

namespace homo {

namespace {

constexpr int TX = 32, TY = 8;                 // vertices per block tile in x, y
constexpr int HX = TX + 2, HY = TY + 2;        // with halo
constexpr int PLANE = HX * HY;                 // halo sites per plane (340)
constexpr int EX = TX + 1, EY = TY + 1;        // element moduli tile
constexpr int EPLANE = EX * EY;                // 297
constexpr int kTiledThreads = TX * TY;         // 256
constexpr int kUSlots = 4, kESlots = 3;
// Each halo site holds its 18 values (6 cases x 3 components) in kCh consecutive floats,
// ordered so that the two cases of a pair are adjacent: channel 6p + 2k + l holds case
// 2p + l, component k. A neighbour's 9 case pairs are then 9 8-byte shared-memory loads
// straight into f32x2 registers; with the 72-byte site stride the 8-byte loads of 16
// consecutive sites fall on distinct banks.
constexpr int kCh = 18;
constexpr int kUPlaneFloats = kCh * PLANE;
constexpr int kEFloats = (kESlots * EPLANE + 1) / 2 * 2;   // keeps the low-part bank 8-byte aligned

__host__ __device__ constexpr int chan(int q) { return 6 * ((q / 3) / 2) + 2 * (q % 3) + (q / 3) % 2; }

static_assert(PLANE > kTiledThreads && PLANE <= 2 * kTiledThreads, "two load sites per thread");
static_assert(EPLANE > kTiledThreads && EPLANE <= 2 * kTiledThreads, "two modulus sites per thread");

// periodic index for a >= -1 (tiles wider than a small grid wrap more than once)
__device__ __forceinline__ int wrapi(int a, int n) { return a < 0 ? a + n : (a >= n ? a % n : a); }

__device__ __forceinline__ void cp_async4(float* smem, const float* gmem) {
  const unsigned s = static_cast<unsigned>(__cvta_generic_to_shared(smem));
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait1() { asm volatile("cp.async.wait_group 1;\n" ::: "memory"); }

// Per-thread load sites (fixed for every plane): halo site tid and, if it exists,
// tid + 256, as in-plane offsets gy*n + gx; same for the moduli tile.
struct Sites {
  int u0, u1;       // in-plane global offsets (u1 < 0: no second site)
  int e0, e1;
};

__device__ __forceinline__ Sites make_sites(int n, int x0, int y0) {
  Sites s;
  const int t = threadIdx.x;
  {
    const int row = t / HX, col = t - row * HX;
    s.u0 = wrapi(y0 - 1 + row, n) * n + wrapi(x0 - 1 + col, n);
  }
  {
    const int k = t + kTiledThreads;
    if (k < PLANE) {
      const int row = k / HX, col = k - row * HX;
      s.u1 = wrapi(y0 - 1 + row, n) * n + wrapi(x0 - 1 + col, n);
    } else {
      s.u1 = -1;
    }
  }
  {
    const int row = t / EX, col = t - row * EX;
    s.e0 = wrapi(y0 - 1 + row, n) * n + wrapi(x0 - 1 + col, n);
  }
  {
    const int k = t + kTiledThreads;
    if (k < EPLANE) {
      const int row = k / EX, col = k - row * EX;
      s.e1 = wrapi(y0 - 1 + row, n) * n + wrapi(x0 - 1 + col, n);
    } else {
      s.e1 = -1;
    }
  }
  return s;
}

__device__ __forceinline__ void issue_u_plane(const float* __restrict__ u, size_t N, size_t zoff,
                                              const Sites& s, float* __restrict__ dst) {
  const float* g = u + zoff;
#pragma unroll
  for (int q = 0; q < kPlanes; ++q) {
    cp_async4(dst + threadIdx.x * kCh + chan(q), g + q * N + s.u0);
    if (s.u1 >= 0) cp_async4(dst + (threadIdx.x + kTiledThreads) * kCh + chan(q), g + q * N + s.u1);
  }
}

__device__ __forceinline__ void issue_e_plane(const float* __restrict__ E, size_t zoff, const Sites& s,
                                              float* __restrict__ dst) {
  cp_async4(dst + threadIdx.x, E + zoff + s.e0);
  if (s.e1 >= 0) cp_async4(dst + threadIdx.x + kTiledThreads, E + zoff + s.e1);
}

// The 9 case pairs of one site: 9 8-byte loads (kCh * 4 = 72 bytes per site: every site,
// slot and bank starts on an 8-byte boundary).
__device__ __forceinline__ void load_pairs(const float* site, f32x2 (&pr)[9]) {
  const unsigned long long* p2 = reinterpret_cast<const unsigned long long*>(site);
#pragma unroll
  for (int i = 0; i < 9; ++i) pr[i] = p2[i];
}

// MODE 1: out = K u in difference form (sum_d A_d (u_(v+d) - u_v)) with partials of the
//         dots (u_c, out_c) and the 18 plane sums of out (the CG product);
// MODE 2: out = b - K (u + ulo) in difference form, each neighbour difference formed from
//         the high and the low parts, (u_(v+d) - u_v) + (ulo_(v+d) - ulo_v), with partials of
//         ||out_c||^2 and the 18 plane sums of out (the true residual of a double-float
//         displacement, in FP32). The high difference is exact or within 2 ulp of the
//         difference itself, so every term carries FP32 relative accuracy and the residual
//         is accurate to ~1e-7 of sum_d |A_d| |u_(v+d) - u_v|; the low parts ride in a
//         second bank of plane slots;
// MODE 3: out = b - K u (the V-cycle residual).
// MODE 4: out = u + c0 S^-1 (b - K u), S the 3x3 diagonal block (first Chebyshev step);
// MODE 5: out = u + c0 (u - out) + c1 S^-1 (b - K u): a later Chebyshev step, the previous
//         iterate read from out and replaced in place;
// MODE 6: out = (1 + c0) u + c1 S^-1 (b - K u): the same step when the previous iterate is 0.
// b is reduced by bmean (plane means) when bmean is non-null (modes 3-5).
template <int MODE>
__global__ void __launch_bounds__(kTiledThreads, MODE == 2 ? 1 : 2)
    k_fine_tiled(const __grid_constant__ KeParam K, const float* __restrict__ E,
                 const float* __restrict__ u, const float* __restrict__ ulo,
                 const float* __restrict__ b, float* out, int n, int zchunk,
                 double* __restrict__ part, const double* __restrict__ bmean, float c0, float c1) {
  constexpr bool kLo = MODE == 2;
  extern __shared__ float sm[];
  float* su = sm;                                   // kUSlots x PLANE x kCh
  float* se = sm + kUSlots * kUPlaneFloats;         // kESlots x EPLANE
  float* sl = se + kEFloats;                        // low parts (MODE 2): kUSlots x PLANE x kCh
  const size_t N = static_cast<size_t>(n) * n * n;
  const size_t nn = static_cast<size_t>(n) * n;
  const int tx = threadIdx.x % TX, ty = threadIdx.x / TX;
  const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
  const int z0 = blockIdx.z * zchunk;
  const int z1 = min(z0 + zchunk, n);
  const int x = x0 + tx, y = y0 + ty;
  const bool live = x < n && y < n;
  const Sites s = make_sites(n, x0, y0);
  float red[kCases + kPlanes];
#pragma unroll
  for (int c = 0; c < kCases + kPlanes; ++c) red[c] = 0.f;

  // prologue: u planes z0-1, z0, z0+1 and modulus planes z0-1, z0
  for (int p = -1; p <= 1; ++p) {
    const int zp = wrapi(z0 + p, n);
    issue_u_plane(u, N, zp * nn, s, su + ((z0 + p + kUSlots) & 3) * kUPlaneFloats);
    if (kLo) issue_u_plane(ulo, N, zp * nn, s, sl + ((z0 + p + kUSlots) & 3) * kUPlaneFloats);
  }
  for (int p = -1; p <= 0; ++p) {
    const int zp = wrapi(z0 + p, n);
    issue_e_plane(E, zp * nn, s, se + ((z0 + p + kESlots) % kESlots) * EPLANE);
  }
  cp_async_commit();

  for (int z = z0; z < z1; ++z) {
    // prefetch u plane z+2 and modulus plane z+1 (their slots were released at the end
    // of the previous step)
    issue_u_plane(u, N, static_cast<size_t>(wrapi(z + 2, n)) * nn, s, su + ((z + 2) & 3) * kUPlaneFloats);
    if (kLo)
      issue_u_plane(ulo, N, static_cast<size_t>(wrapi(z + 2, n)) * nn, s, sl + ((z + 2) & 3) * kUPlaneFloats);
    issue_e_plane(E, static_cast<size_t>(wrapi(z + 1, n)) * nn, s, se + ((z + 1) % kESlots) * EPLANE);
    cp_async_commit();
    cp_async_wait1();
    __syncthreads();
    if (live) {
      const int sm1 = ((z + 3) & 3) * kUPlaneFloats, s0 = (z & 3) * kUPlaneFloats,
                sp1 = ((z + 1) & 3) * kUPlaneFloats;               // planes z-1, z, z+1
      const float* em = se + ((z + 2) % kESlots) * EPLANE;     // elements with origin z-1
      const float* e0 = se + (z % kESlots) * EPLANE;           // elements with origin z
      float Et[8];
#pragma unroll
      for (int t = 0; t < 8; ++t)
        Et[t] = ((t >> 2) ? e0 : em)[(ty + ((t >> 1) & 1)) * EX + tx + (t & 1)];
      const int cidx = (ty + 1) * HX + tx + 1;
      constexpr bool kDiff = MODE == 1 || MODE == 2;
      // the 6 cases advance in pairs (2p, 2p + 1) on the two lanes of f32x2 registers;
      // every lane is rounded as the scalar chain in the same order would be
      constexpr int kPairs = kCases / 2;
      // pair j = 3p + k (cases 2p, 2p + 1, component k) sits at channels 2j, 2j + 1
      f32x2 own[3 * kPairs], ownlo[3 * kPairs];
      if (kDiff) load_pairs(su + s0 + cidx * kCh, own);
      if (kLo) load_pairs(sl + s0 + cidx * kCh, ownlo);
      constexpr bool kCheb = MODE == 4 || MODE == 5 || MODE == 6;
      f32x2 accp[3 * kPairs];
#pragma unroll
      for (int q = 0; q < 3 * kPairs; ++q) accp[q] = 0ull;
      float S[9];
#pragma unroll
      for (int d = 0; d < 27; ++d) {
        if (kDiff && d == 13) continue;
        const int dx = d % 3 - 1, dy = (d / 3) % 3 - 1, dz = d / 9 - 1;
        float A[9];
        nb_block(K, Et, dx, dy, dz, A);
        if (kCheb && d == 13) {
#pragma unroll
          for (int q = 0; q < 9; ++q) S[q] = A[q];
        }
        f32x2 Ap[9];
#pragma unroll
        for (int e = 0; e < 9; ++e) Ap[e] = pack2(A[e], A[e]);
        const int off = (dz < 0 ? sm1 : (dz == 0 ? s0 : sp1)) + (cidx + dy * HX + dx) * kCh;
        f32x2 uv[3 * kPairs];
        load_pairs(su + off, uv);
        if (kDiff) {
#pragma unroll
          for (int j = 0; j < 3 * kPairs; ++j) uv[j] = fsub2(uv[j], own[j]);
        }
        if (kLo) {
          f32x2 lv[3 * kPairs];
          load_pairs(sl + off, lv);
#pragma unroll
          for (int j = 0; j < 3 * kPairs; ++j) uv[j] = fadd2(uv[j], fsub2(lv[j], ownlo[j]));
        }
#pragma unroll
        for (int p = 0; p < kPairs; ++p) {
#pragma unroll
          for (int r = 0; r < 3; ++r)
            accp[3 * p + r] = ffma2(Ap[3 * r], uv[3 * p], ffma2(Ap[3 * r + 1], uv[3 * p + 1],
                                    ffma2(Ap[3 * r + 2], uv[3 * p + 2], accp[3 * p + r])));
        }
      }
      float acc[kPlanes], own1[kDiff ? kPlanes : 1];
#pragma unroll
      for (int p = 0; p < kPairs; ++p)
#pragma unroll
        for (int r = 0; r < 3; ++r) {
          unpack2(accp[3 * p + r], acc[6 * p + r], acc[6 * p + 3 + r]);
          if (kDiff) unpack2(own[3 * p + r], own1[kDiff ? 6 * p + r : 0], own1[kDiff ? 6 * p + 3 + r : 0]);
        }
      const size_t v = static_cast<size_t>(z) * nn + static_cast<size_t>(y) * n + x;
      if (kCheb) {
        // residual, block-diagonal solve, Chebyshev update
#pragma unroll
        for (int q = 0; q < kPlanes; ++q)
          acc[q] = (__ldg(b + q * N + v) - (bmean ? static_cast<float>(bmean[q]) : 0.f)) - acc[q];
        solve3x6(S, acc);
#pragma unroll
        for (int q = 0; q < kPlanes; ++q) {
          const size_t o = q * N + v;
          const float uc = su[s0 + cidx * kCh + chan(q)];
          if (MODE == 4) out[o] = fmaf(c0, acc[q], uc);
          else if (MODE == 5) out[o] = fmaf(c1, acc[q], fmaf(c0, uc - out[o], uc));
          else out[o] = fmaf(c1, acc[q], fmaf(c0, uc, uc));
        }
      } else {
#pragma unroll
        for (int q = 0; q < kPlanes; ++q) {
          const size_t o = q * N + v;
          float val = acc[q];
          if (MODE == 3) val = (__ldg(b + o) - (bmean ? static_cast<float>(bmean[q]) : 0.f)) - val;
          if (MODE == 2) val = __ldg(b + o) - val;
          out[o] = val;
          if (MODE == 1) red[q / 3] = fmaf(own1[kDiff ? q : 0], val, red[q / 3]);
          if (MODE == 2) red[q / 3] = fmaf(val, val, red[q / 3]);
          if (kDiff) red[kCases + q] += val;
        }
      }
    }
    __syncthreads();
  }
  if ((MODE == 1 || MODE == 2) && part != nullptr) {
    // block_sum_store writes row blockIdx.x; shift the base to the flattened 3-D index
    const size_t flat = (static_cast<size_t>(blockIdx.z) * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
    block_sum_store<kCases + kPlanes>(red, part + (flat - blockIdx.x) * (kCases + kPlanes));
  }
}

int tiled_zchunk(int n) {
  // enough blocks for ~8 waves of 2 resident blocks per SM on 152 SMs
  const long xy = static_cast<long>((n + TX - 1) / TX) * ((n + TY - 1) / TY);
  int chunk = n;
  while (chunk > 4 && xy * ((n + chunk - 1) / chunk) < 152L * 2 * 8) chunk = (chunk + 1) / 2;
  return chunk;
}

}  // namespace

size_t tiled_smem_bytes(int mode) {
  return sizeof(float) * (kUSlots * kUPlaneFloats * (mode == 2 ? 2 : 1) + kEFloats);
}

int tiled_grid_blocks(int n) {
  const int zc = tiled_zchunk(n);
  return ((n + TX - 1) / TX) * ((n + TY - 1) / TY) * ((n + zc - 1) / zc);
}

namespace {
template <int MODE>
cudaError_t run_tiled(const homo_ctx* c, dim3 grid, int zc, const float* u, const float* ulo, const float* b,
                      float* out, double* part, const double* bmean, float c0, float c1) {
  const size_t shm = tiled_smem_bytes(MODE);   // limit set by tiled_init at context creation
  k_fine_tiled<MODE><<<grid, kTiledThreads, shm, c->stream>>>(c->ke, c->E, u, ulo, b, out, c->n, zc, part,
                                                              bmean, c0, c1);
  return cudaGetLastError();
}
}  // namespace

template <int MODE>
cudaError_t tiled_attr() {
  return cudaFuncSetAttribute(k_fine_tiled<MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              static_cast<int>(tiled_smem_bytes(MODE)));
}

cudaError_t tiled_init() {
  cudaError_t e = tiled_attr<1>();
  if (e == cudaSuccess) e = tiled_attr<2>();
  if (e == cudaSuccess) e = tiled_attr<3>();
  if (e == cudaSuccess) e = tiled_attr<4>();
  if (e == cudaSuccess) e = tiled_attr<5>();
  if (e == cudaSuccess) e = tiled_attr<6>();
  return e;
}

cudaError_t launch_fine_tiled(const homo_ctx* c, int mode, const float* u, const float* b, float* out,
                              double* part, int* grid_out, const double* bmean, float c0, float c1,
                              const float* ulo) {
  const int n = c->n;
  const int zc = tiled_zchunk(n);
  dim3 grid((n + TX - 1) / TX, (n + TY - 1) / TY, (n + zc - 1) / zc);
  if (grid_out) *grid_out = static_cast<int>(grid.x * grid.y * grid.z);
  switch (mode) {
    case 1: return run_tiled<1>(c, grid, zc, u, nullptr, nullptr, out, part, nullptr, 0.f, 0.f);
    case 2:
      if (!ulo) return cudaErrorInvalidValue;
      return run_tiled<2>(c, grid, zc, u, ulo, b, out, part, nullptr, 0.f, 0.f);
    case 3: return run_tiled<3>(c, grid, zc, u, nullptr, b, out, nullptr, bmean, 0.f, 0.f);
    case 4: return run_tiled<4>(c, grid, zc, u, nullptr, b, out, nullptr, bmean, c0, c1);
    case 5: return run_tiled<5>(c, grid, zc, u, nullptr, b, out, nullptr, bmean, c0, c1);
    case 6: return run_tiled<6>(c, grid, zc, u, nullptr, b, out, nullptr, bmean, c0, c1);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace homo
