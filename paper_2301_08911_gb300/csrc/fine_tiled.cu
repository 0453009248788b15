// Tiled finest-level stencil kernels: each block owns a 32 x 8 column of vertices over a
// chunk of z planes and marches along z. Four planes of the 6-case field (with a
// one-vertex periodic halo) and three planes of element moduli live in shared memory;
// the plane two steps ahead is fetched with asynchronous copies (cp.async) while the
// current plane is computed, so global latency overlaps the arithmetic. Each thread
// builds the 27 coupling blocks A_d of its vertex (Eq. 13) from the moduli and the
// element matrix in the parameter bank and applies them to the 6 load cases.
#include "dev_common.cuh"

namespace homo {

namespace {

constexpr int TX = 32, TY = 8;                 // vertices per block tile in x, y
constexpr int HX = TX + 2, HY = TY + 2;        // with halo
constexpr int PLANE = HX * HY;                 // halo sites per plane (340)
constexpr int EX = TX + 1, EY = TY + 1;        // element moduli tile
constexpr int EPLANE = EX * EY;                // 297
constexpr int kTiledThreads = TX * TY;         // 256
constexpr int kUSlots = 4, kESlots = 3;
constexpr int kUPlaneFloats = kPlanes * PLANE;

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

__device__ __forceinline__ void tile_block(const KeParam& K, const float (&Et)[8], int dx, int dy,
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
    cp_async4(dst + q * PLANE + threadIdx.x, g + q * N + s.u0);
    if (s.u1 >= 0) cp_async4(dst + q * PLANE + threadIdx.x + kTiledThreads, g + q * N + s.u1);
  }
}

__device__ __forceinline__ void issue_e_plane(const float* __restrict__ E, size_t zoff, const Sites& s,
                                              float* __restrict__ dst) {
  cp_async4(dst + threadIdx.x, E + zoff + s.e0);
  if (s.e1 >= 0) cp_async4(dst + threadIdx.x + kTiledThreads, E + zoff + s.e1);
}

// MODE 1: out = K u in difference form (sum_d A_d (u_(v+d) - u_v)) with partials of the
//         dots (u_c, out_c) and the 18 plane sums of out (the CG product);
// MODE 3: out = b - K u (the V-cycle residual).
template <int MODE>
__global__ void __launch_bounds__(kTiledThreads, 2) k_fine_tiled(const __grid_constant__ KeParam K,
                                                                 const float* __restrict__ E,
                                                                 const float* __restrict__ u,
                                                                 const float* __restrict__ b,
                                                                 float* __restrict__ out, int n,
                                                                 int zchunk,
                                                                 double* __restrict__ part) {
  extern __shared__ float sm[];
  float* su = sm;                                   // kUSlots x 18 x PLANE
  float* se = sm + kUSlots * kUPlaneFloats;         // kESlots x EPLANE
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
    issue_e_plane(E, static_cast<size_t>(wrapi(z + 1, n)) * nn, s, se + ((z + 1) % kESlots) * EPLANE);
    cp_async_commit();
    cp_async_wait1();
    __syncthreads();
    if (live) {
      const float* pm = su + ((z + 3) & 3) * kUPlaneFloats;   // plane z-1
      const float* p0 = su + (z & 3) * kUPlaneFloats;         // plane z
      const float* pp = su + ((z + 1) & 3) * kUPlaneFloats;   // plane z+1
      const float* em = se + ((z + 2) % kESlots) * EPLANE;     // elements with origin z-1
      const float* e0 = se + (z % kESlots) * EPLANE;           // elements with origin z
      float Et[8];
#pragma unroll
      for (int t = 0; t < 8; ++t)
        Et[t] = ((t >> 2) ? e0 : em)[(ty + ((t >> 1) & 1)) * EX + tx + (t & 1)];
      const int cidx = (ty + 1) * HX + tx + 1;
      float own[kPlanes];
      if (MODE == 1) {
#pragma unroll
        for (int q = 0; q < kPlanes; ++q) own[q] = p0[q * PLANE + cidx];
      }
      float acc[kPlanes];
#pragma unroll
      for (int q = 0; q < kPlanes; ++q) acc[q] = 0.f;
#pragma unroll
      for (int d = 0; d < 27; ++d) {
        if (MODE == 1 && d == 13) continue;
        const int dx = d % 3 - 1, dy = (d / 3) % 3 - 1, dz = d / 9 - 1;
        float A[9];
        tile_block(K, Et, dx, dy, dz, A);
        const float* p = (dz < 0 ? pm : (dz == 0 ? p0 : pp)) + cidx + dy * HX + dx;
#pragma unroll
        for (int c = 0; c < kCases; ++c) {
          float uu[3];
#pragma unroll
          for (int k = 0; k < 3; ++k) {
            uu[k] = p[(3 * c + k) * PLANE];
            if (MODE == 1) uu[k] -= own[3 * c + k];
          }
#pragma unroll
          for (int r = 0; r < 3; ++r)
            acc[3 * c + r] = fmaf(A[3 * r], uu[0], fmaf(A[3 * r + 1], uu[1], fmaf(A[3 * r + 2], uu[2], acc[3 * c + r])));
        }
      }
      const size_t v = static_cast<size_t>(z) * nn + static_cast<size_t>(y) * n + x;
#pragma unroll
      for (int q = 0; q < kPlanes; ++q) {
        const size_t o = q * N + v;
        float val = acc[q];
        if (MODE == 3) val = __ldg(b + o) - val;
        out[o] = val;
        if (MODE == 1) {
          red[q / 3] = fmaf(own[q], val, red[q / 3]);
          red[kCases + q] += val;
        }
      }
    }
    __syncthreads();
  }
  if (MODE == 1 && part != nullptr) {
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

size_t tiled_smem_bytes() { return sizeof(float) * (kUSlots * kUPlaneFloats + kESlots * EPLANE); }

int tiled_grid_blocks(int n) {
  const int zc = tiled_zchunk(n);
  return ((n + TX - 1) / TX) * ((n + TY - 1) / TY) * ((n + zc - 1) / zc);
}

cudaError_t launch_fine_tiled(const homo_ctx* c, int mode, const float* u, const float* b, float* out,
                              double* part, int* grid_out) {
  const int n = c->n;
  const int zc = tiled_zchunk(n);
  dim3 grid((n + TX - 1) / TX, (n + TY - 1) / TY, (n + zc - 1) / zc);
  if (grid_out) *grid_out = static_cast<int>(grid.x * grid.y * grid.z);
  const size_t shm = tiled_smem_bytes();
  cudaError_t e;
  if (mode == 1) {
    e = cudaFuncSetAttribute(k_fine_tiled<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(shm));
    if (e != cudaSuccess) return e;
    k_fine_tiled<1><<<grid, kTiledThreads, shm, c->stream>>>(c->ke, c->E, u, nullptr, out, n, zc, part);
  } else {
    e = cudaFuncSetAttribute(k_fine_tiled<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(shm));
    if (e != cudaSuccess) return e;
    k_fine_tiled<3><<<grid, kTiledThreads, shm, c->stream>>>(c->ke, c->E, u, b, out, n, zc, nullptr);
  }
  return cudaGetLastError();
}

}  // namespace homo
