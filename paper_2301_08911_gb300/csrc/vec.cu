// Vector kernels of the CG driver, reductions, the periodic density filter and the OC
// update. All reductions are two-stage and deterministic: per-block partials in FP64,
// then one block sums them in a fixed order.
#include <cmath>

#include "dev_common.cuh"

namespace homo {

namespace {

// W consecutive floats (W = 4: one 16-byte access; the caller guarantees alignment, i.e.
// N % 4 == 0 so that every plane starts on a 16-byte boundary).
template <int W>
struct Pk {
  float v[W];
};

template <int W>
__device__ __forceinline__ Pk<W> ldg_pk(const float* __restrict__ p) {
  Pk<W> r;
  if constexpr (W == 4) {
    const float4 t = __ldg(reinterpret_cast<const float4*>(p));
    r.v[0] = t.x; r.v[1] = t.y; r.v[2] = t.z; r.v[3] = t.w;
  } else {
    r.v[0] = __ldg(p);
  }
  return r;
}

template <int W>
__device__ __forceinline__ Pk<W> ld_pk(const float* p) {
  Pk<W> r;
  if constexpr (W == 4) {
    const float4 t = *reinterpret_cast<const float4*>(p);
    r.v[0] = t.x; r.v[1] = t.y; r.v[2] = t.z; r.v[3] = t.w;
  } else {
    r.v[0] = *p;
  }
  return r;
}

template <int W>
__device__ __forceinline__ void st_pk(float* p, const Pk<W>& x) {
  if constexpr (W == 4) *reinterpret_cast<float4*>(p) = make_float4(x.v[0], x.v[1], x.v[2], x.v[3]);
  else *p = x.v[0];
}

// hi + lo += d + dlo in double-float (TwoSum, then FastTwoSum renormalisation), with
// operations the compiler may not contract or reorder.
__device__ __forceinline__ void df_add(float& hi, float& lo, float d, float dlo) {
  const float sm = __fadd_rn(hi, d);
  const float bb = __fadd_rn(sm, -hi);
  const float er = __fadd_rn(__fadd_rn(hi, -__fadd_rn(sm, -bb)), __fadd_rn(d, -bb));
  const float l = __fadd_rn(__fadd_rn(lo, dlo), er);
  const float s2 = __fadd_rn(sm, l);
  lo = __fadd_rn(l, -__fadd_rn(s2, -sm));
  hi = s2;
}

__global__ void __launch_bounds__(256) k_sum_partials(const double* __restrict__ part, int nblk,
                                                      int nv, double* __restrict__ out) {
  // thread t owns value k = t % nv of rows r0, r0 + per, r0 + 2 per, ... (r0 = t / nv):
  // the block reads the row-major partials contiguously, with four independent sums
  __shared__ double sh[256];
  const int t = threadIdx.x;
  const int per = blockDim.x / nv;
  const int k = t % nv, r0 = t / nv;
  double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
  if (r0 < per) {
    const size_t stride = static_cast<size_t>(per) * nv;
    const size_t total = static_cast<size_t>(nblk) * nv;
    size_t i = static_cast<size_t>(r0) * nv + k;
    for (; i + 3 * stride < total; i += 4 * stride) {
      s0 += part[i];
      s1 += part[i + stride];
      s2 += part[i + 2 * stride];
      s3 += part[i + 3 * stride];
    }
    for (; i < total; i += stride) s0 += part[i];
  }
  sh[t] = (s0 + s1) + (s2 + s3);
  __syncthreads();
  if (t < nv) {
    double acc = 0.0;
    for (int r = 0; r < per; ++r) acc += sh[r * nv + t];
    out[t] = acc;
  }
}

// Per case c: sum over the 3 planes of case c of a*b. Each thread takes W consecutive
// vertices per step (W = 4: 16-byte accesses, four times the bytes in flight).
template <int W>
__global__ void __launch_bounds__(256) k_dot6(const float* __restrict__ a,
                                              const float* __restrict__ b, size_t N,
                                              double* __restrict__ part) {
  float red[kCases];
#pragma unroll
  for (int c = 0; c < kCases; ++c) red[c] = 0.f;
  for (size_t i = static_cast<size_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < N / W;
       i += static_cast<size_t>(gridDim.x) * blockDim.x) {
    const size_t v = i * W;
#pragma unroll
    for (int q = 0; q < kPlanes; ++q) {
      const Pk<W> x = ldg_pk<W>(a + q * N + v), y = ldg_pk<W>(b + q * N + v);
#pragma unroll
      for (int w = 0; w < W; ++w) red[q / 3] = fmaf(x.v[w], y.v[w], red[q / 3]);
    }
  }
  block_sum_store<kCases>(red, part);
}

// (r_c - mean r, z_c) for the 6 cases and the 18 plane sums of z (for removing its mean).
// rmean: 18 plane means of r (doubles), or null.
template <int W>
__global__ void __launch_bounds__(256) k_dot6_zsum(const float* __restrict__ r,
                                                   const float* __restrict__ z, size_t N,
                                                   const double* __restrict__ rmean,
                                                   double* __restrict__ part) {
  float red[kCases + kPlanes], rm[kPlanes];
#pragma unroll
  for (int c = 0; c < kCases + kPlanes; ++c) red[c] = 0.f;
#pragma unroll
  for (int q = 0; q < kPlanes; ++q) rm[q] = rmean ? static_cast<float>(rmean[q]) : 0.f;
  for (size_t i = static_cast<size_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < N / W;
       i += static_cast<size_t>(gridDim.x) * blockDim.x) {
    const size_t v = i * W;
#pragma unroll
    for (int q = 0; q < kPlanes; ++q) {
      const Pk<W> zz = ldg_pk<W>(z + q * N + v), rr = ldg_pk<W>(r + q * N + v);
#pragma unroll
      for (int w = 0; w < W; ++w) {
        red[q / 3] = fmaf(rr.v[w] - rm[q], zz.v[w], red[q / 3]);
        red[kCases + q] += zz.v[w];
      }
    }
  }
  block_sum_store<kCases + kPlanes>(red, part);
}

__global__ void k_cg_alpha(double* __restrict__ s) {
  const int c = threadIdx.x;
  if (c >= kCases) return;
  const double pq = s[S_PQ + c];
  double a = 0.0;
  if (s[S_ACTIVE + c] != 0.0 && pq > 0.0 && isfinite(pq)) a = s[S_RZ + c] / pq;
  s[S_ALPHA + c] = a;
}

// beta = rz_new / rz_old (0 on the first step or for finished cases); rz_old <- rz_new.
__global__ void k_cg_beta(double* __restrict__ s, int first) {
  const int c = threadIdx.x;
  if (c >= kCases) return;
  const double rz = s[S_RZ + c], old = s[S_RZ_OLD + c];
  double b = 0.0;
  if (!first && s[S_ACTIVE + c] != 0.0 && old != 0.0 && isfinite(rz)) b = rz / old;
  s[S_BETA + c] = b;
  s[S_RZ_OLD + c] = rz;
}

// The stored residual keeps the plane means it had when it was last recomputed (the
// rigid translations, outside the range of K); every consumer subtracts them. This
// kernel turns the raw sums into the centred norms ||r_c - mean||^2 = sum r^2 - sum^2/N
// and the plane means, and marks case c active while ||r_c||^2 > tol^2 ||f_c||^2.
__global__ void k_cg_active(double* __restrict__ s, double tol2, double N) {
  const int c = threadIdx.x;
  if (c >= kCases) return;
  double rr = s[S_RR + c];
  for (int k = 0; k < 3; ++k) {
    const double sum = s[S_RSUM + 3 * c + k];
    rr -= sum * sum / N;
    s[S_RMEAN + 3 * c + k] = sum / N;
  }
  rr = fmax(rr, 0.0);
  s[S_RR + c] = rr;
  const double ff = s[S_FF + c];
  s[S_ACTIVE + c] = (ff > 0.0 && rr > tol2 * ff) ? 1.0 : 0.0;
}

// e += alpha p, e kept in double-float (e + elo): the product is split exactly (its
// rounding error recovered with an FMA) and both parts are added with error-free
// transformations, so the correction carries no FP32 rounding noise; K applied to such
// noise would be amplified by the operator's spread of eigenvalues and leave the true
// residual far above the recursive one. r -= alpha (q - mean q) in FP32. Partial sums of
// ||r_c||^2 and of the 18 plane sums of r.
template <int W>
__global__ void __launch_bounds__(256) k_cg_update_er(float* __restrict__ e, float* __restrict__ elo,
                                                      float* __restrict__ r,
                                                      const float* __restrict__ p,
                                                      const float* __restrict__ q,
                                                      const double* __restrict__ s, size_t N,
                                                      double* __restrict__ part) {
  float a[kCases];
#pragma unroll
  for (int c = 0; c < kCases; ++c) a[c] = static_cast<float>(s[S_ALPHA + c]);
  float red[kCases + kPlanes], qm[kPlanes];
#pragma unroll
  for (int c = 0; c < kCases + kPlanes; ++c) red[c] = 0.f;
#pragma unroll
  for (int k = 0; k < kPlanes; ++k) qm[k] = static_cast<float>(s[S_QSUM + k] / static_cast<double>(N));
  for (size_t i = static_cast<size_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < N / W;
       i += static_cast<size_t>(gridDim.x) * blockDim.x) {
    const size_t v = i * W;
#pragma unroll
    for (int k = 0; k < kPlanes; ++k) {
      const int c = k / 3;
      const size_t o = static_cast<size_t>(k) * N + v;
      Pk<W> rv = ld_pk<W>(r + o);
      if (a[c] != 0.f) {
        const Pk<W> pv = ldg_pk<W>(p + o), qv = ldg_pk<W>(q + o);
        Pk<W> hi = ld_pk<W>(e + o), lo = ld_pk<W>(elo + o);
#pragma unroll
        for (int w = 0; w < W; ++w) {
          const float pr = __fmul_rn(a[c], pv.v[w]);        // TwoProd: pr + pe = a p exactly
          const float pe = fmaf(a[c], pv.v[w], -pr);
          df_add(hi.v[w], lo.v[w], pr, pe);
          rv.v[w] = fmaf(-a[c], qv.v[w] - qm[k], rv.v[w]);
        }
        st_pk<W>(e + o, hi);
        st_pk<W>(elo + o, lo);
        st_pk<W>(r + o, rv);
      }
#pragma unroll
      for (int w = 0; w < W; ++w) {
        red[c] = fmaf(rv.v[w], rv.v[w], red[c]);
        red[kCases + k] += rv.v[w];
      }
    }
  }
  block_sum_store<kCases + kPlanes>(red, part);
}

// (u + ulo) += (e + elo) in double-float arithmetic (error-free transformations with
// non-contracted operations), then e = elo = 0. Closes a CG cycle. n % W == 0.
template <int W>
__global__ void __launch_bounds__(256) k_fold(float* __restrict__ u, float* __restrict__ ulo,
                                              float* __restrict__ e, float* __restrict__ elo,
                                              size_t n) {
  Pk<W> zero;
#pragma unroll
  for (int w = 0; w < W; ++w) zero.v[w] = 0.f;
  for (size_t i = static_cast<size_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < n / W;
       i += static_cast<size_t>(gridDim.x) * blockDim.x) {
    const size_t o = i * W;
    const Pk<W> d = ld_pk<W>(e + o), dlo = ld_pk<W>(elo + o);
    Pk<W> hi = ld_pk<W>(u + o), lo = ld_pk<W>(ulo + o);
#pragma unroll
    for (int w = 0; w < W; ++w) df_add(hi.v[w], lo.v[w], d.v[w], dlo.v[w]);
    st_pk<W>(u + o, hi);
    st_pk<W>(ulo + o, lo);
    st_pk<W>(e + o, zero);
    st_pk<W>(elo + o, zero);
  }
}

// p = (z - mean(z)) + beta p per plane.
template <int W>
__global__ void __launch_bounds__(256) k_cg_update_p(float* __restrict__ p,
                                                     const float* __restrict__ z,
                                                     const double* __restrict__ s, size_t N) {
  float b[kCases], mz[kPlanes];
#pragma unroll
  for (int c = 0; c < kCases; ++c) b[c] = static_cast<float>(s[S_BETA + c]);
#pragma unroll
  for (int k = 0; k < kPlanes; ++k) mz[k] = static_cast<float>(s[S_ZSUM + k] / static_cast<double>(N));
  for (size_t i = static_cast<size_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < N / W;
       i += static_cast<size_t>(gridDim.x) * blockDim.x) {
    const size_t v = i * W;
#pragma unroll
    for (int k = 0; k < kPlanes; ++k) {
      const size_t o = static_cast<size_t>(k) * N + v;
      const Pk<W> zz = ldg_pk<W>(z + o);
      Pk<W> pp;
      if (b[k / 3] != 0.f) {
        pp = ld_pk<W>(p + o);
#pragma unroll
        for (int w = 0; w < W; ++w) pp.v[w] = fmaf(b[k / 3], pp.v[w], zz.v[w] - mz[k]);
      } else {
#pragma unroll
        for (int w = 0; w < W; ++w) pp.v[w] = zz.v[w] - mz[k];
      }
      st_pk<W>(p + o, pp);
    }
  }
}

__global__ void k_split_set(float* __restrict__ hi, float* __restrict__ lo,
                            const float* __restrict__ src, size_t n) {
  for (size_t i = static_cast<size_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
       i += static_cast<size_t>(gridDim.x) * blockDim.x) {
    hi[i] = src[i];
    lo[i] = 0.f;
  }
}

__global__ void k_split_get(const float* __restrict__ hi, const float* __restrict__ lo,
                            float* __restrict__ dst, size_t n) {
  for (size_t i = static_cast<size_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
       i += static_cast<size_t>(gridDim.x) * blockDim.x)
    dst[i] = hi[i] + lo[i];
}

// Periodic linear-cone filter: out_e = inv_wsum * sum_k w_k in_(e + off_k).
// kSens = false: out_e = sum_d w(d) in_(e+d) / sum_d w(d) (density filter, its own
// adjoint). kSens = true: the density-weighted sensitivity filter of the unfiltered variant
// (Sec. 5.3), out_e = sum_d w(d) rho_(e+d) in_(e+d) / (max(gamma, rho_e) sum_d w(d)).
template <bool kSens>
__global__ void __launch_bounds__(256) k_filter(const __grid_constant__ FilterParam F, int n,
                                                const float* __restrict__ in,
                                                const float* __restrict__ rho, float gamma,
                                                float* __restrict__ out) {
  const size_t N = static_cast<size_t>(n) * n * n;
  for (size_t e = static_cast<size_t>(blockIdx.x) * blockDim.x + threadIdx.x; e < N;
       e += static_cast<size_t>(gridDim.x) * blockDim.x) {
    int x, y, z;
    decode3(static_cast<unsigned>(e), static_cast<unsigned>(n), x, y, z);
    float s = 0.f;
    for (int k = 0; k < F.count; ++k) {
      int xx = x + F.off[k][0], yy = y + F.off[k][1], zz = z + F.off[k][2];
      xx += xx < 0 ? n : (xx >= n ? -n : 0);
      yy += yy < 0 ? n : (yy >= n ? -n : 0);
      zz += zz < 0 ? n : (zz >= n ? -n : 0);
      const size_t f = xx + static_cast<size_t>(n) * (yy + static_cast<size_t>(n) * zz);
      const float v = kSens ? __ldg(in + f) * __ldg(rho + f) : __ldg(in + f);
      s = fmaf(F.w[k], v, s);
    }
    out[e] = kSens ? s * F.inv_wsum / fmaxf(gamma, __ldg(rho + e)) : s * F.inv_wsum;
  }
}

// ---------------------------------------------------------------- OC update
// rho_new(s) = clamp(base_e * s, lo_e, hi_e), base_e = rho_e max(-dc_e, 0)^eta,
// s = lambda^(-eta); mean(rho_new) increases with s. OC scratch (doubles at S_OC):
constexpr int kOcCand = 15;      // candidate multipliers per pass
// kOcPasses passes (homo_internal.cuh): the bracket shrinks 16x per pass in log scale
enum { OC_SLO = 0, OC_SHI = 1, OC_MODE = 2, OC_CAND = 8, OC_CHANGE = 32, OC_SUMS = 40 };

__device__ __forceinline__ float oc_lo(float r, float move, float rmin) { return fmaxf(rmin, r - move); }
__device__ __forceinline__ float oc_hi(float r, float move) { return fminf(1.f, r + move); }

// base -> tmp; block partials [min lo/base, max hi/base, sum lo, sum hi] over base > 0.
__global__ void __launch_bounds__(256) k_oc_setup(const float* __restrict__ rho,
                                                  const float* __restrict__ dc,
                                                  float* __restrict__ base, size_t N, float eta,
                                                  float move, float rmin,
                                                  double* __restrict__ part) {
  float mn = INFINITY, mx = 0.f;
  double slo = 0.0, shi = 0.0;
  for (size_t e = static_cast<size_t>(blockIdx.x) * blockDim.x + threadIdx.x; e < N;
       e += static_cast<size_t>(gridDim.x) * blockDim.x) {
    const float r = rho[e];
    const float D = fmaxf(-dc[e], 0.f);
    const float bs = D > 0.f ? r * powf(D, eta) : 0.f;
    base[e] = bs;
    const float lo = oc_lo(r, move, rmin), hi = oc_hi(r, move);
    slo += lo;
    shi += hi;
    if (bs > 0.f) {
      mn = fminf(mn, lo / bs);
      mx = fmaxf(mx, hi / bs);
    }
  }
  __shared__ float smn[256], smx[256];
  __shared__ double ssl[256], ssh[256];
  smn[threadIdx.x] = mn;
  smx[threadIdx.x] = mx;
  ssl[threadIdx.x] = slo;
  ssh[threadIdx.x] = shi;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) {
      smn[threadIdx.x] = fminf(smn[threadIdx.x], smn[threadIdx.x + o]);
      smx[threadIdx.x] = fmaxf(smx[threadIdx.x], smx[threadIdx.x + o]);
      ssl[threadIdx.x] += ssl[threadIdx.x + o];
      ssh[threadIdx.x] += ssh[threadIdx.x + o];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    double* o = part + 4 * static_cast<size_t>(blockIdx.x);
    o[0] = smn[0];
    o[1] = smx[0];
    o[2] = ssl[0];
    o[3] = ssh[0];
  }
}

__device__ void oc_make_candidates(double* oc) {
  const double lo = oc[OC_SLO], hi = oc[OC_SHI];
  const double lr = log(hi / lo);
  for (int k = 0; k < kOcCand; ++k) oc[OC_CAND + k] = lo * exp(lr * (k + 1) / (kOcCand + 1));
}

__global__ void k_oc_setup_final(const double* __restrict__ part, int nblk, size_t N, double V,
                                 double* __restrict__ oc) {
  if (threadIdx.x != 0) return;
  double mn = INFINITY, mx = 0.0, sl = 0.0, sh = 0.0;
  for (int b = 0; b < nblk; ++b) {
    mn = fmin(mn, part[4 * b]);
    mx = fmax(mx, part[4 * b + 1]);
    sl += part[4 * b + 2];
    sh += part[4 * b + 3];
  }
  const double vlo = sl / static_cast<double>(N), vhi = sh / static_cast<double>(N);
  oc[OC_SLO] = mn;
  oc[OC_SHI] = mx;
  if (!(mx > 0.0) || !isfinite(mn) || vlo >= V) oc[OC_MODE] = 2;     // everything at its lower bound
  else if (vhi <= V) oc[OC_MODE] = 1;                                // everything at its upper bound
  else oc[OC_MODE] = 0;
  if (oc[OC_MODE] == 0) oc_make_candidates(oc);
}

__global__ void __launch_bounds__(256) k_oc_pass(const float* __restrict__ rho,
                                                 const float* __restrict__ base, size_t N,
                                                 float move, float rmin,
                                                 const double* __restrict__ oc,
                                                 double* __restrict__ part) {
  if (oc[OC_MODE] != 0) return;
  float cand[kOcCand], acc[kOcCand];
  double accd[kOcCand];
#pragma unroll
  for (int k = 0; k < kOcCand; ++k) {
    cand[k] = static_cast<float>(oc[OC_CAND + k]);
    acc[k] = 0.f;
    accd[k] = 0.0;
  }
  int cnt = 0;
  for (size_t e = static_cast<size_t>(blockIdx.x) * blockDim.x + threadIdx.x; e < N;
       e += static_cast<size_t>(gridDim.x) * blockDim.x) {
    const float r = __ldg(rho + e), bs = __ldg(base + e);
    const float lo = oc_lo(r, move, rmin), hi = oc_hi(r, move);
#pragma unroll
    for (int k = 0; k < kOcCand; ++k) acc[k] += fminf(fmaxf(bs * cand[k], lo), hi);
    if (++cnt == 8) {   // FP32 over at most 8 terms, FP64 beyond
#pragma unroll
      for (int k = 0; k < kOcCand; ++k) {
        accd[k] += acc[k];
        acc[k] = 0.f;
      }
      cnt = 0;
    }
  }
#pragma unroll
  for (int k = 0; k < kOcCand; ++k) accd[k] += acc[k];
  block_sum_store_d<kOcCand>(accd, part);
}

// sums: the kOcCand volume sums already reduced over blocks.
__global__ void k_oc_pass_final(const double* __restrict__ sums, size_t N, double V,
                                double* __restrict__ oc) {
  if (threadIdx.x != 0 || oc[OC_MODE] != 0) return;
  double lo = oc[OC_SLO], hi = oc[OC_SHI];
  for (int k = 0; k < kOcCand; ++k) {
    const double vol = sums[k] / static_cast<double>(N);
    if (vol <= V) {
      lo = oc[OC_CAND + k];
    } else {
      hi = oc[OC_CAND + k];
      break;
    }
  }
  oc[OC_SLO] = lo;
  oc[OC_SHI] = hi;
  oc_make_candidates(oc);
}

__global__ void __launch_bounds__(256) k_oc_apply(float* __restrict__ rho,
                                                  const float* __restrict__ base, size_t N,
                                                  float move, float rmin,
                                                  const double* __restrict__ oc,
                                                  double* __restrict__ part) {
  const int mode = static_cast<int>(oc[OC_MODE]);
  const float s = mode == 2 ? 0.f : static_cast<float>(mode == 1 ? oc[OC_SHI] : oc[OC_SLO]);
  float ch = 0.f;
  for (size_t e = static_cast<size_t>(blockIdx.x) * blockDim.x + threadIdx.x; e < N;
       e += static_cast<size_t>(gridDim.x) * blockDim.x) {
    const float r = rho[e];
    const float lo = oc_lo(r, move, rmin), hi = oc_hi(r, move);
    const float nr = fminf(fmaxf(base[e] * s, lo), hi);
    ch = fmaxf(ch, fabsf(nr - r));
    rho[e] = nr;
  }
  __shared__ float sm[256];
  sm[threadIdx.x] = ch;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) sm[threadIdx.x] = fmaxf(sm[threadIdx.x], sm[threadIdx.x + o]);
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = sm[0];
}

__global__ void k_max_partials(const double* __restrict__ part, int nblk, double* __restrict__ out) {
  if (threadIdx.x != 0) return;
  double m = 0.0;
  for (int b = 0; b < nblk; ++b) m = fmax(m, part[b]);
  *out = m;
}

// Orbit averages under a cube symmetry group (Sec. 6.1). Thread per element: it forms
// the indices of the element's images (index arithmetic only) and continues only if its
// own index is the smallest, i.e. once per orbit; that thread sums the orbit's values in
// FP64 and writes the average to every member. For values within a factor 2^29 of each
// other (densities in [1e-3, 1], say) the FP64 sum of at most 48 FP32 values is exact, so
// the result does not depend on the order and every member gets the same FP32 value.
// Orbits are disjoint, so the kernel may run in place.
__device__ __forceinline__ unsigned sym_image(const SymParam& S, int g, int x, int y, int z, int n) {
  const int c[3] = {x, y, z};
  int j[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const int p = S.perm[g][k];
    const int v = p == 0 ? c[0] : (p == 1 ? c[1] : c[2]);
    j[k] = ((S.flip[g] >> k) & 1) ? n - 1 - v : v;
  }
  return static_cast<unsigned>(j[0]) + static_cast<unsigned>(n) * (j[1] + static_cast<unsigned>(n) * j[2]);
}

__global__ void __launch_bounds__(256) k_symmetrize(const __grid_constant__ SymParam S, const float* in,
                                                    float* out, int n) {
  const unsigned N = static_cast<unsigned>(n) * n * n;
  for (unsigned e = blockIdx.x * blockDim.x + threadIdx.x; e < N; e += gridDim.x * blockDim.x) {
    int x, y, z;
    decode3(e, static_cast<unsigned>(n), x, y, z);
    bool canonical = true;
    for (int g = 0; g < S.count && canonical; ++g) canonical = sym_image(S, g, x, y, z, n) >= e;
    if (!canonical) continue;
    double acc = 0.0;
    for (int g = 0; g < S.count; ++g) acc += static_cast<double>(in[sym_image(S, g, x, y, z, n)]);
    const float avg = static_cast<float>(acc / S.count);
    for (int g = 0; g < S.count; ++g) out[sym_image(S, g, x, y, z, n)] = avg;
  }
}

// Trigonometric initialisation (Sec. 6.2), FP64 throughout (a one-time setup step).
// Basis order: T index 2 (3 (k - 1) + i) + {0: cos, 1: sin} of 2 pi k xb_i, then the
// products T_a T_b, a <= b, row by row; xb = R (centre - 1/2).
__global__ void __launch_bounds__(256) k_trig_basis(const __grid_constant__ TrigParam P, int n, double* y) {
  const unsigned N = static_cast<unsigned>(n) * n * n;
  const int nt = 6 * P.nb;
  for (unsigned e = blockIdx.x * blockDim.x + threadIdx.x; e < N; e += gridDim.x * blockDim.x) {
    int x, yy, z;
    decode3(e, static_cast<unsigned>(n), x, yy, z);
    const double c[3] = {(x + 0.5) / n - 0.5, (yy + 0.5) / n - 0.5, (z + 0.5) / n - 0.5};
    double xb[3];
    for (int r = 0; r < 3; ++r) xb[r] = P.R[3 * r] * c[0] + P.R[3 * r + 1] * c[1] + P.R[3 * r + 2] * c[2];
    double T[kTrigMaxT];
    for (int k = 1; k <= P.nb; ++k)
      for (int i = 0; i < 3; ++i) {
        double sv, cv;
        sincospi(2.0 * k * xb[i], &sv, &cv);
        T[2 * (3 * (k - 1) + i)] = cv;
        T[2 * (3 * (k - 1) + i) + 1] = sv;
      }
    double acc = 0.0;
    int idx = 0;
    for (int a = 0; a < nt; ++a) acc = fma(P.w[idx++], T[a], acc);
    for (int a = 0; a < nt; ++a)
      for (int b = a; b < nt; ++b) acc = fma(P.w[idx++], T[a] * T[b], acc);
    y[e] = acc;
  }
}

__device__ __forceinline__ double trig_sigmoid(double y, double mu, double k, double Vh, double rho_min) {
  const double r = rho_min + Vh / (1.0 + exp(-k * (y - mu)));
  return fmin(fmax(r, rho_min), 1.0);
}

__global__ void __launch_bounds__(256) k_trig_volume(const double* __restrict__ y, size_t N, double mu0,
                                                     double dmu, double k, double Vh, double rho_min,
                                                     double* __restrict__ part) {
  double acc[kTrigCand];
#pragma unroll
  for (int c = 0; c < kTrigCand; ++c) acc[c] = 0.0;
  for (size_t e = static_cast<size_t>(blockIdx.x) * blockDim.x + threadIdx.x; e < N;
       e += static_cast<size_t>(gridDim.x) * blockDim.x) {
    const double v = y[e];
#pragma unroll
    for (int c = 0; c < kTrigCand; ++c) acc[c] += trig_sigmoid(v, mu0 + c * dmu, k, Vh, rho_min);
  }
  block_sum_store_d<kTrigCand>(acc, part);
}

__global__ void __launch_bounds__(256) k_trig_project(const double* __restrict__ y, size_t N, double mu,
                                                      double k, double Vh, double rho_min, float* rho) {
  for (size_t e = static_cast<size_t>(blockIdx.x) * blockDim.x + threadIdx.x; e < N;
       e += static_cast<size_t>(gridDim.x) * blockDim.x)
    rho[e] = static_cast<float>(trig_sigmoid(y[e], mu, k, Vh, rho_min));
}

}  // namespace

int reduce_grid(size_t n_items) { return grid_for(n_items, 256); }

cudaError_t launch_sum_partials(const double* part, int nblk, int nv, double* out,
                                cudaStream_t s) {
  if (nv < 1 || nv > 256) return cudaErrorInvalidValue;
  k_sum_partials<<<1, 256, 0, s>>>(part, nblk, nv, out);
  return cudaGetLastError();
}

cudaError_t launch_dot6(const float* a, const float* b, size_t N, double* part, int* grid_out,
                        cudaStream_t s) {
  const int g = grid_for(N % 4 == 0 ? N / 4 : N, 256);
  *grid_out = g;
  if (N % 4 == 0) k_dot6<4><<<g, 256, 0, s>>>(a, b, N, part);
  else k_dot6<1><<<g, 256, 0, s>>>(a, b, N, part);
  return cudaGetLastError();
}

cudaError_t launch_dot6_zsum(const float* r, const float* z, size_t N, const double* rmean,
                             double* part, int* grid_out, cudaStream_t s) {
  const int g = grid_for(N % 4 == 0 ? N / 4 : N, 256);
  *grid_out = g;
  if (N % 4 == 0) k_dot6_zsum<4><<<g, 256, 0, s>>>(r, z, N, rmean, part);
  else k_dot6_zsum<1><<<g, 256, 0, s>>>(r, z, N, rmean, part);
  return cudaGetLastError();
}

cudaError_t launch_cg_alpha(double* scal, cudaStream_t s) {
  k_cg_alpha<<<1, 32, 0, s>>>(scal);
  return cudaGetLastError();
}

cudaError_t launch_cg_beta(double* scal, int first, cudaStream_t s) {
  k_cg_beta<<<1, 32, 0, s>>>(scal, first);
  return cudaGetLastError();
}

cudaError_t launch_cg_active(double* scal, double tol, size_t N, cudaStream_t s) {
  k_cg_active<<<1, 32, 0, s>>>(scal, tol * tol, static_cast<double>(N));
  return cudaGetLastError();
}

cudaError_t launch_cg_update_er(float* e, float* elo, float* r, const float* p, const float* q,
                                const double* scal, size_t N, double* part, int* grid_out,
                                cudaStream_t s) {
  const int g = grid_for(N % 4 == 0 ? N / 4 : N, 256);
  *grid_out = g;
  if (N % 4 == 0) k_cg_update_er<4><<<g, 256, 0, s>>>(e, elo, r, p, q, scal, N, part);
  else k_cg_update_er<1><<<g, 256, 0, s>>>(e, elo, r, p, q, scal, N, part);
  return cudaGetLastError();
}

cudaError_t launch_fold(float* u, float* ulo, float* e, float* elo, size_t n, cudaStream_t s) {
  if (n % 4 == 0) k_fold<4><<<grid_for(n / 4, 256), 256, 0, s>>>(u, ulo, e, elo, n);
  else k_fold<1><<<grid_for(n, 256), 256, 0, s>>>(u, ulo, e, elo, n);
  return cudaGetLastError();
}

cudaError_t launch_cg_update_p(float* p, const float* z, const double* scal, size_t N,
                               cudaStream_t s) {
  if (N % 4 == 0) k_cg_update_p<4><<<grid_for(N / 4, 256), 256, 0, s>>>(p, z, scal, N);
  else k_cg_update_p<1><<<grid_for(N, 256), 256, 0, s>>>(p, z, scal, N);
  return cudaGetLastError();
}

cudaError_t launch_split_set(float* hi, float* lo, const float* src, size_t n, cudaStream_t s) {
  k_split_set<<<grid_for(n, 256), 256, 0, s>>>(hi, lo, src, n);
  return cudaGetLastError();
}

cudaError_t launch_split_get(const float* hi, const float* lo, float* dst, size_t n,
                             cudaStream_t s) {
  k_split_get<<<grid_for(n, 256), 256, 0, s>>>(hi, lo, dst, n);
  return cudaGetLastError();
}

int build_sym_param(int kind, SymParam& sp) {
  sp.count = 0;
  const int perms[6][3] = {{0, 1, 2}, {0, 2, 1}, {1, 0, 2}, {1, 2, 0}, {2, 0, 1}, {2, 1, 0}};
  const int parity[6] = {1, -1, -1, 1, 1, -1};
  if (kind != HOMO_SYM_REFLECT3 && kind != HOMO_SYM_ROTATE3 && kind != HOMO_SYM_REFLECT6) return HOMO_EINVAL;
  for (int p = 0; p < 6; ++p)
    for (int f = 0; f < 8; ++f) {
      const int det = parity[p] * (((f & 1) + ((f >> 1) & 1) + (f >> 2)) % 2 ? -1 : 1);
      if (kind == HOMO_SYM_REFLECT3 && p != 0) continue;
      if (kind == HOMO_SYM_ROTATE3 && det != 1) continue;
      for (int k = 0; k < 3; ++k) sp.perm[sp.count][k] = static_cast<unsigned char>(perms[p][k]);
      sp.flip[sp.count] = static_cast<unsigned char>(f);
      ++sp.count;
    }
  return HOMO_OK;
}

cudaError_t launch_trig_basis(const TrigParam& tp, int n, double* y, cudaStream_t s) {
  const size_t N = static_cast<size_t>(n) * n * n;
  k_trig_basis<<<grid_for(N, 256), 256, 0, s>>>(tp, n, y);
  return cudaGetLastError();
}

cudaError_t launch_trig_volume(const double* y, size_t N, double mu0, double dmu, double k, double Vh,
                               double rho_min, double* part, int* grid_out, cudaStream_t s) {
  const int g = grid_for(N, 256);
  *grid_out = g;
  k_trig_volume<<<g, 256, 0, s>>>(y, N, mu0, dmu, k, Vh, rho_min, part);
  return cudaGetLastError();
}

cudaError_t launch_trig_project(const double* y, size_t N, double mu, double k, double Vh, double rho_min,
                                float* rho, cudaStream_t s) {
  k_trig_project<<<grid_for(N, 256), 256, 0, s>>>(y, N, mu, k, Vh, rho_min, rho);
  return cudaGetLastError();
}

cudaError_t launch_symmetrize(const SymParam& sp, int n, const float* in, float* out, cudaStream_t s) {
  const size_t N = static_cast<size_t>(n) * n * n;
  k_symmetrize<<<grid_for(N, 256), 256, 0, s>>>(sp, in, out, n);
  return cudaGetLastError();
}

cudaError_t launch_filter(const FilterParam& fp, int n, const float* in, float* out,
                          cudaStream_t s) {
  const size_t N = static_cast<size_t>(n) * n * n;
  k_filter<false><<<grid_for(N, 256), 256, 0, s>>>(fp, n, in, nullptr, 0.f, out);
  return cudaGetLastError();
}

cudaError_t launch_sensitivity_filter(const FilterParam& fp, int n, const float* rho, const float* dc,
                                      float gamma, float* out, cudaStream_t s) {
  const size_t N = static_cast<size_t>(n) * n * n;
  k_filter<true><<<grid_for(N, 256), 256, 0, s>>>(fp, n, dc, rho, gamma, out);
  return cudaGetLastError();
}

cudaError_t launch_oc(homo_ctx* c, const float* dc, float* rho, double volfrac, double move,
                      double eta, double rho_min, double* change) {
  const size_t N = c->N;
  const int g = grid_for(N, 256);
  double* oc = c->scal + S_OC;
  cudaStream_t s = c->stream;
  k_oc_setup<<<g, 256, 0, s>>>(rho, dc, c->tmp, N, static_cast<float>(eta), static_cast<float>(move),
                               static_cast<float>(rho_min), c->part);
  k_oc_setup_final<<<1, 32, 0, s>>>(c->part, g, N, volfrac, oc);
  for (int it = 0; it < kOcPasses; ++it) {
    k_oc_pass<<<g, 256, 0, s>>>(rho, c->tmp, N, static_cast<float>(move), static_cast<float>(rho_min), oc,
                                c->part);
    k_sum_partials<<<1, 256, 0, s>>>(c->part, g, kOcCand, oc + OC_SUMS);
    k_oc_pass_final<<<1, 32, 0, s>>>(oc + OC_SUMS, N, volfrac, oc);
  }
  k_oc_apply<<<g, 256, 0, s>>>(rho, c->tmp, N, static_cast<float>(move), static_cast<float>(rho_min), oc,
                               c->part);
  k_max_partials<<<1, 32, 0, s>>>(c->part, g, oc + OC_CHANGE);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  if (change) {
    e = cudaMemcpyAsync(c->hscal + S_OC + OC_CHANGE, oc + OC_CHANGE, sizeof(double),
                        cudaMemcpyDeviceToHost, s);
    if (e != cudaSuccess) return e;
    e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return e;
    *change = c->hscal[S_OC + OC_CHANGE];
  }
  return cudaSuccess;
}

}  // namespace homo
