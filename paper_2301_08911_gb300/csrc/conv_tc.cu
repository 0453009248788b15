// Periodic 3x3x3 convolution of the warm-start network on the 5th-generation tensor cores
// (tcgen05.mma, accumulators in tensor memory). Implicit GEMM: M = 128 voxels, N = 32
// output channels, K = 27 taps x c_in, BF16 operands, FP32 accumulation.
//
// A persistent CTA (4 warps) keeps the layer's weights in shared memory and walks tiles of
// 30 x 4 x 2 output voxels. Each tile's periodic halo box (32 x 6 x 4 voxels, all input
// channels) is staged with 16-byte asynchronous copies into a K-major, non-swizzled
// operand layout whose rows are 16 bytes apart along the box's (z, y, x) order: channel
// chunk c (8 channels) of box row r sits at plane c, row r. For a tap with offset d, the
// 128 rows of the A operand are then the output rows shifted by the constant row offset of
// d, so every tap's operand is the same staged box seen through a shifted descriptor, with
// no per-tap copy. Output rows 0 and 31 of each 32-row run are halo positions: computed and
// discarded (30 of every 32 rows are outputs).
//
// One thread issues the tile's 27 x c_in/16 MMAs per output plane into two 32-column TMEM
// accumulators and commits them to an mbarrier; after a bounded wait every warp reads its
// 32 TMEM lanes (one voxel per thread, 32 channels) and applies the same epilogues as the
// other layers: bias, residual, ReLU or a backward ReLU mask, BF16 voxel-major output or
// scaled FP32 displacement planes.
#include <cuda_bf16.h>

#include <algorithm>
#include <cstdint>
#include <cstring>

#include "dev_common.cuh"

namespace homo {
namespace {

constexpr int kC = HOMO_NN_CHANNELS;     // 32 output channels
constexpr int kTaps = 27;
constexpr int TXo = 30, TYo = 4, TZo = 2;                 // output voxels per tile
constexpr int BXr = TXo + 2, BYr = TYo + 2, BZr = TZo + 2; // box (32 x 6 x 4)
constexpr int kBoxRows = BXr * BYr * BZr;                  // 768
constexpr int kRowPad = 1;                                 // row 0: guard below the box
constexpr int kRows = 776;                                 // >= kRowPad + kBoxRows + 1, multiple of 8
constexpr int kPlaneBytes = kRows * 16;                    // one 8-channel chunk of every row
constexpr int kThreads = 128;
constexpr int kTmemCols = 64;                              // two 128 x 32 FP32 accumulators
constexpr long long kWaitLimit = 1LL << 18;                // bounded mbarrier polls (~1 s on a GB300)

static_assert(kRowPad + kBoxRows + 1 <= kRows, "guard rows");
static_assert(kThreads == 4 * 32 && TYo == 4, "warp w owns output row y = w of each plane");

template <int CIN>
struct TcShape {
  static constexpr int kChunks = CIN / 8;
  static constexpr int kBoxBytes = kChunks * kPlaneBytes;
  static constexpr int kWBytes = kTaps * kChunks * kC * 16;
  static constexpr int kBytes = kBoxBytes + kWBytes + 64;   // + mbarrier and TMEM address
};

struct TcScale {
  float s[6];
};

__device__ int g_conv_tc_timeouts = 0;   // tiles whose MMA completion wait ran out

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void cp_async16(uint32_t dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(dst), "l"(src) : "memory");
}

__device__ __forceinline__ int wrapc(int a, int n) {
  a %= n;
  return a < 0 ? a + n : a;
}

// Shared-memory matrix descriptor of a K-major, non-swizzled operand: core matrices of
// 8 rows x 16 bytes with rows 16 bytes apart, 8-row groups SBO bytes apart along M/N and
// 16-byte K chunks LBO bytes apart; descriptor version 1 (bits 46-47), no base offset.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= static_cast<uint64_t>((addr & 0x3FFFFu) >> 4);
  d |= static_cast<uint64_t>((lbo >> 4) & 0x3FFFu) << 16;
  d |= static_cast<uint64_t>((sbo >> 4) & 0x3FFFu) << 32;
  d |= static_cast<uint64_t>(1) << 46;
  return d;   // layout type 0 (no swizzle) in bits 61-63
}

// Instruction descriptor of kind::f16: FP32 accumulator, BF16 A and B, both K-major,
// N = 32, M = 128.
constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((kC >> 3) << 17) | ((128 >> 4) << 24);

__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem_d),
      "l"(a), "l"(b), "r"(kIdesc), "r"(accumulate));
}

__device__ __forceinline__ void mma_commit(uint32_t mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(mbar)
               : "memory");
}

// Poll the mbarrier for phase `parity` at most kWaitLimit times; true once it completed.
__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t parity) {
  for (long long i = 0; i < kWaitLimit; ++i) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(done)
        : "r"(mbar), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];\n"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
        "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]),
        "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]),
        "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ uint32_t bf2(float a, float b) {
  const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);   // a -> low half
  uint32_t u;
  memcpy(&u, &h, 4);
  return u;
}

__device__ __forceinline__ float2 unbf2(uint32_t u) {
  __nv_bfloat162 h;
  memcpy(&h, &u, 4);
  return __bfloat1622float2(h);
}

template <int CIN, int EPI>
__global__ void __launch_bounds__(kThreads, 2)
    k_conv3d_tc(int n, int tiles_x, int tiles_y, int ntiles, const __nv_bfloat16* __restrict__ x,
                const __nv_bfloat16* __restrict__ w, const float* __restrict__ bias,
                const __nv_bfloat16* __restrict__ res, const __nv_bfloat16* __restrict__ mask,
                __nv_bfloat16* __restrict__ out, float* __restrict__ outf, TcScale sc) {
  using S = TcShape<CIN>;
  constexpr int kCh = S::kChunks;
  extern __shared__ __align__(128) unsigned char smem[];
  unsigned char* box = smem;                              // kCh planes x kRows x 16 B
  unsigned char* wsm = smem + S::kBoxBytes;               // [tap][chunk][o][16 B]
  uint64_t* mbar = reinterpret_cast<uint64_t*>(smem + S::kBoxBytes + S::kWBytes);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(mbar + 1);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const size_t N = static_cast<size_t>(n) * n * n;
  const uint32_t box_s = smem_u32(box), w_s = smem_u32(wsm), mbar_s = smem_u32(mbar);

  // weights once per CTA; guard rows of every plane zeroed once (never loaded)
  for (int c = tid; c < kTaps * kC * kCh; c += kThreads) {
    const int ch = c % kCh, o = (c / kCh) % kC, tap = c / (kCh * kC);
    cp_async16(w_s + ((tap * kCh + ch) * kC + o) * 16, w + (static_cast<size_t>(tap) * kC + o) * CIN + ch * 8);
  }
  asm volatile("cp.async.commit_group;\n" ::: "memory");
  for (int c = tid; c < kCh * (kRows - kBoxRows); c += kThreads) {
    const int ch = c / (kRows - kBoxRows), r = c % (kRows - kBoxRows);
    const int row = r < kRowPad ? r : kRowPad + kBoxRows + (r - kRowPad);
    *reinterpret_cast<uint4*>(box + ch * kPlaneBytes + row * 16) = make_uint4(0u, 0u, 0u, 0u);
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(mbar_s) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(tmem_slot)),
                 "r"(kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  const uint32_t tmem = *tmem_slot;

  // this thread's TMEM lane (warp w reads lanes 32 w .. 32 w + 31) and output position
  const uint32_t tlane = tmem + (static_cast<uint32_t>(32 * warp) << 16);
  const bool xout = lane >= 1 && lane <= TXo;             // rows 0 and 31 of a run are halo
  float bo[kC], so[18];
#pragma unroll
  for (int o = 0; o < kC; ++o) bo[o] = (EPI != HOMO_NN_MASK && bias) ? bias[o] : 0.f;
#pragma unroll
  for (int o = 0; o < 18; ++o) so[o] = sc.s[o / 3];

  uint32_t phase = 0;
  bool timed_out = false;
  for (int tile = blockIdx.x; tile < ntiles && !timed_out; tile += gridDim.x) {
    const int tx = tile % tiles_x, rest = tile / tiles_x;
    const int ty = rest % tiles_y, tz = rest / tiles_y;
    const int x0 = tx * TXo, y0 = ty * TYo, z0 = tz * TZo;
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();   // the previous tile's TMEM reads and box reads are finished
    for (int c = tid; c < kBoxRows * kCh; c += kThreads) {
      const int ch = c % kCh, br = c / kCh;
      const int bx = br % BXr, by = (br / BXr) % BYr, bz = br / (BXr * BYr);
      const size_t gv = static_cast<size_t>(wrapc(x0 - 1 + bx, n)) +
                        static_cast<size_t>(n) * (wrapc(y0 - 1 + by, n) + static_cast<size_t>(n) * wrapc(z0 - 1 + bz, n));
      cp_async16(box_s + ch * kPlaneBytes + (kRowPad + br) * 16, x + gv * CIN + ch * 8);
    }
    asm volatile("cp.async.commit_group;\n" ::: "memory");
    asm volatile("cp.async.wait_group 0;\n" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");   // copies visible to the tensor core
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    if (tid == 0) {
#pragma unroll 1
      for (int zo = 0; zo < TZo; ++zo) {
        const int r0 = ((zo + 1) * BYr + 1) * BXr;     // box row of output (x = -1, y = 0, z = zo)
#pragma unroll 1
        for (int tap = 0; tap < kTaps; ++tap) {
          const int dx = tap % 3 - 1, dy = (tap / 3) % 3 - 1, dz = tap / 9 - 1;
          const int row = kRowPad + r0 + (dz * BYr + dy) * BXr + dx;
#pragma unroll
          for (int ks = 0; ks < CIN / 16; ++ks) {
            const uint64_t a = smem_desc(box_s + (2 * ks) * kPlaneBytes + row * 16, kPlaneBytes, 128);
            const uint64_t b = smem_desc(w_s + (tap * kCh + 2 * ks) * kC * 16, kC * 16, 128);
            mma_bf16(tmem + zo * kC, a, b, (tap | ks) != 0 ? 1u : 0u);
          }
        }
      }
      mma_commit(mbar_s);
    }
    __syncwarp();
    const bool ok = mbar_wait(mbar_s, phase);
    phase ^= 1u;
    if (__syncthreads_or(!ok)) {         // every thread takes the same decision
      if (tid == 0) atomicAdd(&g_conv_tc_timeouts, 1);
      timed_out = true;
      break;
    }
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
#pragma unroll 1
    for (int zo = 0; zo < TZo; ++zo) {
      float acc[32];
      tmem_ld32(tlane + zo * kC, acc);
      const int gx = x0 + lane - 1, gy = y0 + warp, gz = z0 + zo;
      if (!xout || gx >= n || gy >= n || gz >= n) continue;
      const size_t v = static_cast<size_t>(gx) + static_cast<size_t>(n) * (gy + static_cast<size_t>(n) * gz);
      if (EPI == HOMO_NN_PLANES || EPI == HOMO_NN_PLANES_ADD) {
#pragma unroll
        for (int o = 0; o < 18; ++o) {
          float* d = outf + static_cast<size_t>(o) * N + v;
          const float val = so[o] * (acc[o] + bo[o]);
          *d = EPI == HOMO_NN_PLANES_ADD ? *d + val : val;
        }
        continue;
      }
      uint32_t pk[16];
      const uint4* rp = res ? reinterpret_cast<const uint4*>(res + v * kC) : nullptr;
      const uint4* mp = EPI == HOMO_NN_MASK ? reinterpret_cast<const uint4*>(mask + v * kC) : nullptr;
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        uint32_t rr[4] = {0u, 0u, 0u, 0u}, mm[4] = {0u, 0u, 0u, 0u};
        if (rp) {
          const uint4 t = rp[q];
          rr[0] = t.x; rr[1] = t.y; rr[2] = t.z; rr[3] = t.w;
        }
        if (mp) {
          const uint4 t = mp[q];
          mm[0] = t.x; mm[1] = t.y; mm[2] = t.z; mm[3] = t.w;
        }
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const int o = 8 * q + 2 * j;
          float v0 = acc[o] + bo[o], v1 = acc[o + 1] + bo[o + 1];
          if (rp) {
            const float2 r = unbf2(rr[j]);
            v0 += r.x;
            v1 += r.y;
          }
          if (EPI == HOMO_NN_RELU) {
            v0 = fmaxf(v0, 0.f);
            v1 = fmaxf(v1, 0.f);
          } else {
            const float2 m = unbf2(mm[j]);
            v0 = m.x > 0.f ? v0 : 0.f;
            v1 = m.y > 0.f ? v1 : 0.f;
          }
          pk[4 * q + j] = bf2(v0, v1);
        }
      }
      uint4* dst = reinterpret_cast<uint4*>(out + v * kC);
#pragma unroll
      for (int q = 0; q < 4; ++q) dst[q] = make_uint4(pk[4 * q], pk[4 * q + 1], pk[4 * q + 2], pk[4 * q + 3]);
    }
  }
  if (timed_out) {
    // the tile's MMAs may still be running: give them one more bounded wait before TMEM is freed
    mbar_wait(mbar_s, phase ^ 1u);
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(kTmemCols) : "memory");
  }
}

// The bounded completion wait on an mbarrier that no one arrives on: every CTA gives up
// after kWaitLimit polls and counts the timeout, the path a tile takes when its MMAs never
// complete (no MMA is issued here, so nothing is left in flight).
__global__ void k_wait_probe() {
  __shared__ __align__(8) uint64_t bar;
  const uint32_t b = smem_u32(&bar);
  if (threadIdx.x == 0) asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(b) : "memory");
  __syncthreads();
  const bool ok = mbar_wait(b, 0);
  if (__syncthreads_or(!ok) && threadIdx.x == 0) atomicAdd(&g_conv_tc_timeouts, 1);
}

int g_sms = 0;

int sm_count() {
  if (g_sms == 0) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&g_sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || g_sms < 1)
      g_sms = 152;
  }
  return g_sms;
}

template <int CIN, int EPI>
cudaError_t tc_launch(int n, const void* x, const void* w, const float* bias, const void* res, const void* mask,
                      void* out, float* outf, const double* scale, cudaStream_t s) {
  TcScale sc;
  for (int k = 0; k < 6; ++k) sc.s[k] = scale ? static_cast<float>(scale[k]) : 1.f;
  using S = TcShape<CIN>;
  auto kern = k_conv3d_tc<CIN, EPI>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, S::kBytes);
  if (e != cudaSuccess) return e;
  const int tiles_x = (n + TXo - 1) / TXo, tiles_y = (n + TYo - 1) / TYo, tiles_z = (n + TZo - 1) / TZo;
  const long long ntiles = static_cast<long long>(tiles_x) * tiles_y * tiles_z;
  const int grid = static_cast<int>(std::min<long long>(ntiles, 2LL * sm_count()));
  kern<<<grid, kThreads, S::kBytes, s>>>(n, tiles_x, tiles_y, static_cast<int>(ntiles),
                                         static_cast<const __nv_bfloat16*>(x), static_cast<const __nv_bfloat16*>(w),
                                         bias, static_cast<const __nv_bfloat16*>(res),
                                         static_cast<const __nv_bfloat16*>(mask), static_cast<__nv_bfloat16*>(out),
                                         outf, sc);
  return cudaGetLastError();
}

}  // namespace

// tcgen05 convolution for c_in in {16, 32} and every epilogue (the contract of
// homo_nn_conv3d).
cudaError_t conv3d_tc(int n, int cin, int epi, const void* x, const void* w, const float* bias, const void* res,
                      const void* mask, void* out, float* outf, const double* scale, cudaStream_t s) {
#define HOMO_TC_CASE(CI, EP) \
  if (cin == CI && epi == EP) return tc_launch<CI, EP>(n, x, w, bias, res, mask, out, outf, scale, s);
  HOMO_TC_CASE(16, HOMO_NN_RELU)
  HOMO_TC_CASE(32, HOMO_NN_RELU)
  HOMO_TC_CASE(32, HOMO_NN_MASK)
  HOMO_TC_CASE(32, HOMO_NN_PLANES)
  HOMO_TC_CASE(32, HOMO_NN_PLANES_ADD)
#undef HOMO_TC_CASE
  return cudaErrorInvalidValue;
}

cudaError_t conv3d_tc_wait_probe(int blocks) {
  k_wait_probe<<<blocks, 32>>>();
  const cudaError_t e = cudaGetLastError();
  return e != cudaSuccess ? e : cudaDeviceSynchronize();
}

// Number of tiles whose completion wait ran out since the last call (and reset it).
int conv3d_tc_take_timeouts() {
  int h = 0;
  if (cudaMemcpyFromSymbol(&h, g_conv_tc_timeouts, sizeof(int)) != cudaSuccess) return -1;
  const int zero = 0;
  if (cudaMemcpyToSymbol(g_conv_tc_timeouts, &zero, sizeof(int)) != cudaSuccess) return -1;
  return h;
}

}  // namespace homo
