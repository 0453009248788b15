// Device helpers shared by the kernel translation units: periodic neighbour indexing,
// colour-blocked stencil positions and deterministic block reductions.
#pragma once

#include "homo_internal.cuh"

namespace homo {

constexpr int kGridCap = 152 * 16;   // 152 SMs on GB300, 16 resident 256-thread CTAs max

// (i, j, k) of a linear index m = i + h (j + h k) in 32-bit arithmetic (m < 2^32: every
// grid here has at most 1024^3 vertices): two divisions, remainders by products.
__device__ __forceinline__ void decode3(unsigned m, unsigned h, int& i, int& j, int& k) {
  const unsigned q = m / h;
  const unsigned kk = q / h;
  i = static_cast<int>(m - q * h);
  j = static_cast<int>(q - kk * h);
  k = static_cast<int>(kk);
}

// Wrapped coordinates x-1, x, x+1 premultiplied by the axis stride.
struct Nb {
  int X[3];
  int Y[3];
  int Z[3];
};

__device__ __forceinline__ Nb make_nb(int x, int y, int z, int n) {
  Nb nb;
  const int nn = n * n;
  nb.X[0] = x == 0 ? n - 1 : x - 1;
  nb.X[1] = x;
  nb.X[2] = x == n - 1 ? 0 : x + 1;
  nb.Y[0] = (y == 0 ? n - 1 : y - 1) * n;
  nb.Y[1] = y * n;
  nb.Y[2] = (y == n - 1 ? 0 : y + 1) * n;
  nb.Z[0] = (z == 0 ? n - 1 : z - 1) * nn;
  nb.Z[1] = z * nn;
  nb.Z[2] = (z == n - 1 ? 0 : z + 1) * nn;
  return nb;
}

// Position of vertex (x,y,z) inside a stencil plane: grouped by colour
// (x&1) + 2(y&1) + 4(z&1) when n is even, x-fastest otherwise.
__device__ __forceinline__ size_t stencil_pos(int x, int y, int z, int n, bool cb) {
  if (!cb) return static_cast<size_t>(x) + static_cast<size_t>(n) * (y + static_cast<size_t>(n) * z);
  const int h = n >> 1;
  const int col = (x & 1) | ((y & 1) << 1) | ((z & 1) << 2);
  return static_cast<size_t>(col) * h * h * h + (x >> 1) +
         static_cast<size_t>(h) * ((y >> 1) + static_cast<size_t>(h) * (z >> 1));
}

__device__ __forceinline__ void vertex_of_pos(size_t p, int n, bool cb, int& x, int& y, int& z) {
  if (!cb) {
    x = static_cast<int>(p % n);
    y = static_cast<int>((p / n) % n);
    z = static_cast<int>(p / (static_cast<size_t>(n) * n));
    return;
  }
  const int h = n >> 1;
  const size_t hh = static_cast<size_t>(h) * h * h;
  const int col = static_cast<int>(p / hh);
  const size_t m = p - col * hh;
  x = 2 * static_cast<int>(m % h) + (col & 1);
  y = 2 * static_cast<int>((m / h) % h) + ((col >> 1) & 1);
  z = 2 * static_cast<int>(m / (static_cast<size_t>(h) * h)) + (col >> 2);
}

// Sum NV per-thread float values over the block (warp shuffles in FP32, across warps
// in FP64) and store them at out[blockIdx.x * NV + k]. Fixed order: deterministic.
template <int NV>
__device__ __forceinline__ void block_sum_store(const float (&v)[NV], double* out) {
  __shared__ double sh[32][NV];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int nw = (blockDim.x + 31) >> 5;
#pragma unroll
  for (int k = 0; k < NV; ++k) {
    float s = v[k];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if (lane == 0) sh[wid][k] = static_cast<double>(s);
  }
  __syncthreads();
  for (int k = threadIdx.x; k < NV; k += blockDim.x) {
    double s = 0.0;
    for (int w = 0; w < nw; ++w) s += sh[w][k];
    out[static_cast<size_t>(blockIdx.x) * NV + k] = s;
  }
}

// Same with per-thread FP64 inputs.
template <int NV>
__device__ __forceinline__ void block_sum_store_d(const double (&v)[NV], double* out) {
  __shared__ double sh[32][NV];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int nw = (blockDim.x + 31) >> 5;
#pragma unroll
  for (int k = 0; k < NV; ++k) {
    double s = v[k];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if (lane == 0) sh[wid][k] = s;
  }
  __syncthreads();
  for (int k = threadIdx.x; k < NV; k += blockDim.x) {
    double s = 0.0;
    for (int w = 0; w < nw; ++w) s += sh[w][k];
    out[static_cast<size_t>(blockIdx.x) * NV + k] = s;
  }
}

inline int grid_for(size_t items, int block) {
  size_t g = (items + block - 1) / block;
  if (g > static_cast<size_t>(kGridCap)) g = kGridCap;
  if (g < 1) g = 1;
  return static_cast<int>(g);
}

}  // namespace homo
