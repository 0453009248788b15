// Learned warm start: a periodic 3x3x3 convolution network that maps the filtered
// density of a cell to the 18 displacement planes of its 6 load cases (not part of the
// paper's method, which warm-starts from the previous iterate, Sec. 3.3).
//
// The layers' forward and backward-data convolutions run on the tcgen05 tensor cores
// (conv_tc.cu). This file holds the rest of the network's arithmetic: the weight gradient,
// which contracts over voxels (per tap and voxel chunk a CTA stages the transposed
// operands and accumulates a 32 x c_in block with BF16 mma.sync, FP32 accumulation; a
// second kernel sums the chunks in a fixed order, so it is deterministic), the input
// features, pooling, the MSE loss and its gradient, Adam, and the BF16 weight packing.
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <string>
#include <vector>

#include "dev_common.cuh"

namespace homo {
namespace {

constexpr int kC = HOMO_NN_CHANNELS;    // output channels of every layer (32)
constexpr int kTaps = 27;


__device__ __forceinline__ uint32_t ld32(const __nv_bfloat16* p) {
  return *reinterpret_cast<const uint32_t*>(p);
}
__device__ __forceinline__ uint32_t pack2(float a, float b) {
  const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);   // a -> low half
  uint32_t u;
  memcpy(&u, &h, 4);
  return u;
}

// D = A B + D, A 16x16 row-major, B 16x8 column-major, BF16 in, FP32 accumulate.
__device__ __forceinline__ void mma16816(float* d, const uint32_t* a, uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

__device__ __forceinline__ int wrapc(int a, int n) {
  a %= n;
  return a < 0 ? a + n : a;
}

constexpr int kWgTile = 128;              // voxels per staged weight-gradient tile
constexpr int kWgS = kWgTile + 8;         // bf16 per staged channel row (68 words: 4 mod 32)

// Partial weight gradient of one tap over one chunk of voxel tiles:
// part[(chunk * 27 + tap)][o][i] = sum_v dy[v, o] x[wrap(v + d_tap), i]; the centre-tap
// blocks also sum dy over the chunk for the bias gradient (partb[chunk][o]).
template <int CIN>
__global__ void __launch_bounds__(128)
    k_wgrad(int n, int ntiles, int tiles_per_chunk, const __nv_bfloat16* __restrict__ x,
            const __nv_bfloat16* __restrict__ dy, float* __restrict__ part, float* __restrict__ partb) {
  __shared__ __align__(16) __nv_bfloat16 dys[kC * kWgS];
  __shared__ __align__(16) __nv_bfloat16 xs[CIN * kWgS];
  __shared__ float red[4][kC * CIN];
  const int tap = blockIdx.y, chunk = blockIdx.x;
  const int ddx = tap % 3 - 1, ddy = (tap / 3) % 3 - 1, ddz = tap / 9 - 1;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int g = lane >> 2, t4 = lane & 3;
  const size_t N = static_cast<size_t>(n) * n * n;
  constexpr int NT = CIN / 8;

  float acc[2][NT][4];
#pragma unroll
  for (int mt = 0; mt < 2; ++mt)
#pragma unroll
    for (int nt = 0; nt < NT; ++nt)
#pragma unroll
      for (int q = 0; q < 4; ++q) acc[mt][nt][q] = 0.f;
  float bsum = 0.f;

  const int t_begin = chunk * tiles_per_chunk;
  const int t_end = min(ntiles, t_begin + tiles_per_chunk);
  for (int tile = t_begin; tile < t_end; ++tile) {
    __syncthreads();
    const size_t v = static_cast<size_t>(tile) * kWgTile + tid;   // this thread's voxel
    if (v < N) {
      const uint4* src = reinterpret_cast<const uint4*>(dy + v * kC);
#pragma unroll
      for (int q = 0; q < kC / 8; ++q) {
        const uint4 u = src[q];
        const __nv_bfloat16* e = reinterpret_cast<const __nv_bfloat16*>(&u);
#pragma unroll
        for (int j = 0; j < 8; ++j) dys[(8 * q + j) * kWgS + tid] = e[j];
      }
      const int gx = static_cast<int>(v % n), gy = static_cast<int>((v / n) % n),
                gz = static_cast<int>(v / (static_cast<size_t>(n) * n));
      const size_t vs = static_cast<size_t>(wrapc(gx + ddx, n)) +
                        static_cast<size_t>(n) * (wrapc(gy + ddy, n) + static_cast<size_t>(n) * wrapc(gz + ddz, n));
      const uint4* xsrc = reinterpret_cast<const uint4*>(x + vs * CIN);
#pragma unroll
      for (int q = 0; q < CIN / 8; ++q) {
        const uint4 u = xsrc[q];
        const __nv_bfloat16* e = reinterpret_cast<const __nv_bfloat16*>(&u);
#pragma unroll
        for (int j = 0; j < 8; ++j) xs[(8 * q + j) * kWgS + tid] = e[j];
      }
    } else {
      const __nv_bfloat16 z = __float2bfloat16(0.f);
      for (int c = 0; c < kC; ++c) dys[c * kWgS + tid] = z;
      for (int c = 0; c < CIN; ++c) xs[c * kWgS + tid] = z;
    }
    __syncthreads();
#pragma unroll
    for (int ks = 0; ks < 2; ++ks) {
      const int kb = 32 * warp + 16 * ks;
      uint32_t a[2][4];
#pragma unroll
      for (int mt = 0; mt < 2; ++mt) {
        const __nv_bfloat16* r = dys + (16 * mt + g) * kWgS + kb + 2 * t4;
        a[mt][0] = ld32(r);
        a[mt][1] = ld32(r + 8 * kWgS);
        a[mt][2] = ld32(r + 8);
        a[mt][3] = ld32(r + 8 * kWgS + 8);
      }
#pragma unroll
      for (int nt = 0; nt < NT; ++nt) {
        const __nv_bfloat16* r = xs + (8 * nt + g) * kWgS + kb + 2 * t4;
        const uint32_t b0 = ld32(r), b1 = ld32(r + 8);
        mma16816(acc[0][nt], a[0], b0, b1);
        mma16816(acc[1][nt], a[1], b0, b1);
      }
    }
    if (tap == 13 && tid < kC) {
      for (int j = 0; j < kWgTile; ++j) bsum += __bfloat162float(dys[tid * kWgS + j]);
    }
  }
#pragma unroll
  for (int mt = 0; mt < 2; ++mt)
#pragma unroll
    for (int nt = 0; nt < NT; ++nt) {
      const int o = 16 * mt + g, i = 8 * nt + 2 * t4;
      red[warp][o * CIN + i] = acc[mt][nt][0];
      red[warp][o * CIN + i + 1] = acc[mt][nt][1];
      red[warp][(o + 8) * CIN + i] = acc[mt][nt][2];
      red[warp][(o + 8) * CIN + i + 1] = acc[mt][nt][3];
    }
  __syncthreads();
  float* dst = part + (static_cast<size_t>(chunk) * kTaps + tap) * (kC * CIN);
  for (int e = tid; e < kC * CIN; e += 128) dst[e] = ((red[0][e] + red[1][e]) + red[2][e]) + red[3][e];
  if (tap == 13 && tid < kC) partb[static_cast<size_t>(chunk) * kC + tid] = bsum;
}

// dw[t][o][i] = sum over chunks (in order) of the partials; db[o] likewise.
__global__ void k_wgrad_reduce(int chunks, int per, const float* __restrict__ part,
                               const float* __restrict__ partb, float* __restrict__ dw, float* __restrict__ db) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e < kTaps * per) {
    const int tap = e / per, r = e - tap * per;
    double s = 0.0;
    for (int c = 0; c < chunks; ++c) s += part[(static_cast<size_t>(c) * kTaps + tap) * per + r];
    dw[e] = static_cast<float>(s);
  } else if (e < kTaps * per + kC) {
    const int o = e - kTaps * per;
    double s = 0.0;
    for (int c = 0; c < chunks; ++c) s += partb[static_cast<size_t>(c) * kC + o];
    db[o] = static_cast<float>(s);
  }
}

// x[v] = (rho, rho^2, rho^3, 0 ... 0) in BF16, 16 channels.
__global__ void k_features(size_t N, const float* __restrict__ rho, __nv_bfloat16* __restrict__ x) {
  for (size_t v = blockIdx.x * static_cast<size_t>(blockDim.x) + threadIdx.x; v < N;
       v += static_cast<size_t>(gridDim.x) * blockDim.x) {
    const float r = rho[v];
    uint4 lo, hi;
    lo.x = pack2(r, r * r);
    lo.y = pack2(r * r * r, 0.f);
    lo.z = lo.w = 0u;
    hi.x = hi.y = hi.z = hi.w = 0u;
    uint4* d = reinterpret_cast<uint4*>(x + v * HOMO_NN_FEATURES);
    d[0] = lo;
    d[1] = hi;
  }
}

// Loss sum_{v,p<18} (y[p][v] - u[p][v] inv[p/3])^2 / (18 N) per block (FP64) and the
// BF16 gradient dy[v][p] = 2 (y - u inv) / (18 N), zero in channels 18..31.
struct CaseInv {
  double inv[6];
};

__global__ void __launch_bounds__(256) k_mse(size_t N, const float* __restrict__ y, const float* __restrict__ u,
                                             CaseInv ci, __nv_bfloat16* __restrict__ dy, double* __restrict__ part) {
  __shared__ double sh[256];
  const double w = 2.0 / (18.0 * static_cast<double>(N));
  double s = 0.0;
  for (size_t v = blockIdx.x * static_cast<size_t>(blockDim.x) + threadIdx.x; v < N;
       v += static_cast<size_t>(gridDim.x) * blockDim.x) {
    uint32_t pk[16];
#pragma unroll
    for (int p = 0; p < 18; p += 2) {
      const double e0 = static_cast<double>(y[p * N + v]) - static_cast<double>(u[p * N + v]) * ci.inv[p / 3];
      const double e1 =
          static_cast<double>(y[(p + 1) * N + v]) - static_cast<double>(u[(p + 1) * N + v]) * ci.inv[(p + 1) / 3];
      s += e0 * e0 + e1 * e1;
      pk[p / 2] = pack2(static_cast<float>(w * e0), static_cast<float>(w * e1));
    }
#pragma unroll
    for (int q = 9; q < 16; ++q) pk[q] = 0u;
    uint4* d = reinterpret_cast<uint4*>(dy + v * kC);
#pragma unroll
    for (int q = 0; q < 4; ++q) d[q] = make_uint4(pk[4 * q], pk[4 * q + 1], pk[4 * q + 2], pk[4 * q + 3]);
  }
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = sh[0] / (18.0 * static_cast<double>(N));
}

// out[c] = mean of rho over the f^3 fine voxels of coarse voxel c (grid n -> n / f).
__global__ void k_pool(int n, int f, const float* __restrict__ rho, float* __restrict__ out) {
  const int nc = n / f;
  const size_t Nc = static_cast<size_t>(nc) * nc * nc;
  for (size_t c = blockIdx.x * static_cast<size_t>(blockDim.x) + threadIdx.x; c < Nc;
       c += static_cast<size_t>(gridDim.x) * blockDim.x) {
    const int i = static_cast<int>(c % nc), j = static_cast<int>((c / nc) % nc),
              k = static_cast<int>(c / (static_cast<size_t>(nc) * nc));
    double s = 0.0;
    for (int dz = 0; dz < f; ++dz)
      for (int dy = 0; dy < f; ++dy) {
        const float* row = rho + static_cast<size_t>(i) * f +
                           static_cast<size_t>(n) * (static_cast<size_t>(j) * f + dy + static_cast<size_t>(n) * (static_cast<size_t>(k) * f + dz));
        for (int dx = 0; dx < f; ++dx) s += row[dx];
      }
    out[c] = static_cast<float>(s / (static_cast<double>(f) * f * f));
  }
}

__global__ void k_adam(size_t count, float* __restrict__ w, const float* __restrict__ g, float* __restrict__ m,
                       float* __restrict__ v, float lr, float b1, float b2, float c1, float c2, float eps) {
  for (size_t i = blockIdx.x * static_cast<size_t>(blockDim.x) + threadIdx.x; i < count;
       i += static_cast<size_t>(gridDim.x) * blockDim.x) {
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    w[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
  }
}

// wf[t][o][i] = bf16(w[t][o][i]); wb[t][i][o] = bf16(w[26 - t][o][i]) (weights of the
// transposed convolution that propagates gradients back, when c_in = 32).
__global__ void k_pack(int cin, const float* __restrict__ w, __nv_bfloat16* __restrict__ wf,
                       __nv_bfloat16* __restrict__ wb) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= kTaps * kC * cin) return;
  const int t = e / (kC * cin), r = e - t * kC * cin, o = r / cin, i = r - o * cin;
  const __nv_bfloat16 h = __float2bfloat16_rn(w[e]);
  wf[e] = h;
  if (wb) wb[(static_cast<size_t>(kTaps - 1 - t) * cin + i) * kC + o] = h;
}

int g_num_sms = 0;

int num_sms() {
  if (g_num_sms == 0) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&g_num_sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || g_num_sms < 1)
      g_num_sms = 152;
  }
  return g_num_sms;
}

bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

struct WgradPlan {
  int ntiles, tiles_per_chunk, chunks;
};

WgradPlan wgrad_plan(int n) {
  const size_t N = static_cast<size_t>(n) * n * n;
  WgradPlan p;
  p.ntiles = static_cast<int>((N + kWgTile - 1) / kWgTile);
  const int want = std::max(1, std::min(p.ntiles, 4 * num_sms() / 3));
  p.tiles_per_chunk = (p.ntiles + want - 1) / want;
  p.chunks = (p.ntiles + p.tiles_per_chunk - 1) / p.tiles_per_chunk;
  return p;
}

size_t wgrad_scratch_floats(int n, int cin) {
  const WgradPlan p = wgrad_plan(n);
  return static_cast<size_t>(p.chunks) * (static_cast<size_t>(kTaps) * kC * cin + kC);
}

}  // namespace

// ---- launchers --------------------------------------------------------------------------
cudaError_t nn_conv3d(int n, int cin, const void* x, const void* w, const float* bias, const void* res,
                      const void* mask, int epi, void* out, float* outf, const double* scale, cudaStream_t s) {
  return conv3d_tc(n, cin, epi, x, w, bias, res, mask, out, outf, scale, s);
}

cudaError_t nn_wgrad(int n, int cin, const void* x, const void* dy, float* dw, float* db, float* scratch,
                     cudaStream_t s) {
  const WgradPlan p = wgrad_plan(n);
  float* part = scratch;
  float* partb = scratch + static_cast<size_t>(p.chunks) * kTaps * kC * cin;
  const dim3 grid(p.chunks, kTaps);
  if (cin == 16)
    k_wgrad<16><<<grid, 128, 0, s>>>(n, p.ntiles, p.tiles_per_chunk, static_cast<const __nv_bfloat16*>(x),
                                     static_cast<const __nv_bfloat16*>(dy), part, partb);
  else if (cin == 32)
    k_wgrad<32><<<grid, 128, 0, s>>>(n, p.ntiles, p.tiles_per_chunk, static_cast<const __nv_bfloat16*>(x),
                                     static_cast<const __nv_bfloat16*>(dy), part, partb);
  else
    return cudaErrorInvalidValue;
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const int total = kTaps * kC * cin + kC;
  k_wgrad_reduce<<<(total + 255) / 256, 256, 0, s>>>(p.chunks, kC * cin, part, partb, dw, db);
  return cudaGetLastError();
}

cudaError_t nn_features(int n, const float* rho, void* x, cudaStream_t s) {
  const size_t N = static_cast<size_t>(n) * n * n;
  k_features<<<grid_for(N, 256), 256, 0, s>>>(N, rho, static_cast<__nv_bfloat16*>(x));
  return cudaGetLastError();
}

cudaError_t nn_mse(int n, const float* y, const float* u, const double* scale, void* dy, double* part, int* nblk,
                   cudaStream_t s) {
  CaseInv ci;
  for (int k = 0; k < 6; ++k) ci.inv[k] = 1.0 / scale[k];
  const size_t N = static_cast<size_t>(n) * n * n;
  const int g = std::min(grid_for(N, 256), HOMO_NN_MSE_SCRATCH - 1);
  *nblk = g;
  k_mse<<<g, 256, 0, s>>>(N, y, u, ci, static_cast<__nv_bfloat16*>(dy), part);
  return cudaGetLastError();
}

cudaError_t nn_pool(int n, int f, const float* rho, float* out, cudaStream_t s) {
  const int nc = n / f;
  k_pool<<<grid_for(static_cast<size_t>(nc) * nc * nc, 256), 256, 0, s>>>(n, f, rho, out);
  return cudaGetLastError();
}

cudaError_t nn_adam(size_t count, float* w, const float* g, float* m, float* v, int step, double lr, double b1,
                    double b2, double eps, cudaStream_t s) {
  const double c1 = 1.0 - std::pow(b1, step), c2 = 1.0 - std::pow(b2, step);
  k_adam<<<grid_for(count, 256), 256, 0, s>>>(count, w, g, m, v, static_cast<float>(lr), static_cast<float>(b1),
                                              static_cast<float>(b2), static_cast<float>(c1), static_cast<float>(c2),
                                              static_cast<float>(eps));
  return cudaGetLastError();
}

cudaError_t nn_pack(int cin, const float* w, void* wf, void* wb, cudaStream_t s) {
  const int total = kTaps * kC * cin;
  k_pack<<<(total + 255) / 256, 256, 0, s>>>(cin, w, static_cast<__nv_bfloat16*>(wf),
                                             static_cast<__nv_bfloat16*>(wb));
  return cudaGetLastError();
}

}  // namespace homo

// ---- C ABI ------------------------------------------------------------------------------
using namespace homo;

namespace {

int cuda_status(cudaError_t e) { return e == cudaSuccess ? HOMO_OK : HOMO_ECUDA; }

bool conv_args_ok(int n, int c_in, const void* x, const void* w, const void* res, const void* mask, int epi,
                  const void* out, const float* outf) {
  if (n < 1 || n > 1024 || !x || !w || !aligned16(x) || !aligned16(w)) return false;
  if (res && (reinterpret_cast<uintptr_t>(res) & 3u)) return false;
  switch (epi) {
    case HOMO_NN_RELU:
      return (c_in == 16 || c_in == 32) && out && !mask && !outf && !(reinterpret_cast<uintptr_t>(out) & 3u);
    case HOMO_NN_MASK:
      return c_in == 32 && out && mask && !outf && !(reinterpret_cast<uintptr_t>(out) & 3u) &&
             !(reinterpret_cast<uintptr_t>(mask) & 3u);
    case HOMO_NN_PLANES:
    case HOMO_NN_PLANES_ADD:
      return c_in == 32 && outf && !out && !res && !mask;
    default:
      return false;
  }
}

}  // namespace

extern "C" {

int homo_nn_tc_timeouts(void) { return conv3d_tc_take_timeouts(); }

int homo_nn_tc_wait_probe(int blocks) {
  if (blocks < 1 || blocks > 1024) return HOMO_EINVAL;
  return cuda_status(conv3d_tc_wait_probe(blocks));
}

int homo_nn_conv3d(int n, int c_in, const void* x, const void* w, const float* bias, const void* res,
                   const void* mask, int epilogue, void* out, float* out_planes, const double* scale,
                   void* stream) {
  if (!conv_args_ok(n, c_in, x, w, res, mask, epilogue, out, out_planes)) return HOMO_EINVAL;
  return cuda_status(nn_conv3d(n, c_in, x, w, bias, res, mask, epilogue, out, out_planes, scale,
                               static_cast<cudaStream_t>(stream)));
}

size_t homo_nn_wgrad_scratch(int n, int c_in) {
  if (n < 1 || n > 1024 || (c_in != 16 && c_in != 32)) return 0;
  return wgrad_scratch_floats(n, c_in);
}

int homo_nn_wgrad(int n, int c_in, const void* x, const void* dy, float* dw, float* db, float* scratch,
                  size_t scratch_floats, void* stream) {
  if (n < 1 || n > 1024 || (c_in != 16 && c_in != 32) || !x || !dy || !dw || !db || !scratch) return HOMO_EINVAL;
  if (!aligned16(x) || !aligned16(dy) || scratch_floats < wgrad_scratch_floats(n, c_in)) return HOMO_EINVAL;
  return cuda_status(nn_wgrad(n, c_in, x, dy, dw, db, scratch, static_cast<cudaStream_t>(stream)));
}

int homo_nn_features(int n, const float* rho, void* x, void* stream) {
  if (n < 1 || n > 1024 || !rho || !x || !aligned16(x)) return HOMO_EINVAL;
  return cuda_status(nn_features(n, rho, x, static_cast<cudaStream_t>(stream)));
}

int homo_nn_pool(int n, int factor, const float* rho, float* out, void* stream) {
  if (n < 1 || n > 1024 || factor < 1 || n % factor != 0 || !rho || !out) return HOMO_EINVAL;
  return cuda_status(nn_pool(n, factor, rho, out, static_cast<cudaStream_t>(stream)));
}

static bool scales_ok(const double* scale) {
  if (!scale) return false;
  for (int k = 0; k < 6; ++k)
    if (!(scale[k] > 0.0) || !std::isfinite(scale[k])) return false;
  return true;
}

int homo_nn_mse(int n, const float* y, const float* u, const double* scale, void* dy, double* loss, void* stream) {
  if (n < 1 || n > 1024 || !y || !u || !dy || !loss || !aligned16(dy) || !scales_ok(scale)) return HOMO_EINVAL;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int nblk = 0;
  cudaError_t e = nn_mse(n, y, u, scale, dy, loss + 1, &nblk, s);
  if (e == cudaSuccess) e = launch_sum_partials(loss + 1, nblk, 1, loss, s);
  return cuda_status(e);
}

int homo_nn_adam(size_t count, float* w, const float* g, float* m, float* v, int step, double lr, double beta1,
                 double beta2, double eps, void* stream) {
  if (!w || !g || !m || !v || step < 1 || !(lr >= 0.0) || !(beta1 >= 0.0 && beta1 < 1.0) ||
      !(beta2 >= 0.0 && beta2 < 1.0) || !(eps > 0.0))
    return HOMO_EINVAL;
  if (count == 0) return HOMO_OK;
  return cuda_status(nn_adam(count, w, g, m, v, step, lr, beta1, beta2, eps, static_cast<cudaStream_t>(stream)));
}

int homo_nn_pack(int c_in, const float* w, void* w_fwd, void* w_bwd, void* stream) {
  if ((c_in != 16 && c_in != 32) || !w || !w_fwd || (w_bwd && c_in != 32)) return HOMO_EINVAL;
  return cuda_status(nn_pack(c_in, w, w_fwd, w_bwd, static_cast<cudaStream_t>(stream)));
}

}  // extern "C"
