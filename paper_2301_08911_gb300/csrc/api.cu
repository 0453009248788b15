// C ABI of the library (include/homo.h): context life cycle, the multigrid-preconditioned
// CG driver for the 6 cell problems, C^H, sensitivities, filter and OC update.
#include <algorithm>
#include <array>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <string>

#include "homo_internal.cuh"

using namespace homo;

namespace {

thread_local std::string g_create_err;

int set_err(homo_ctx* c, int code, const std::string& msg) {
  if (c) c->err = msg;
  else g_create_err = msg;
  return code;
}

int cuda_err(homo_ctx* c, cudaError_t e, const char* what) {
  std::string m = std::string(what) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")";
  return set_err(c, e == cudaErrorMemoryAllocation ? HOMO_ENOMEM : HOMO_ECUDA, m);
}

#define CK(ctx, call)                                      \
  do {                                                     \
    cudaError_t e_ = (call);                               \
    if (e_ != cudaSuccess) return cuda_err(ctx, e_, #call); \
  } while (0)

#define RET(x)                      \
  do {                              \
    int r_ = (x);                   \
    if (r_ != HOMO_OK) return r_;   \
  } while (0)

template <typename T>
int dalloc(homo_ctx* c, T** p, size_t count, const char* what) {
  cudaError_t e = cudaMalloc(reinterpret_cast<void**>(p), count * sizeof(T));
  if (e != cudaSuccess) {
    *p = nullptr;
    return cuda_err(c, e, what);
  }
  return HOMO_OK;
}

void free_all(homo_ctx* c) {
  auto f = [](void* p) {
    if (p) cudaFree(p);
  };
  f(c->rho); f(c->E); f(c->u); f(c->ulo); f(c->f); f(c->flo); f(c->r); f(c->z); f(c->pv); f(c->q);
  f(c->tmp); f(c->A); f(c->G); f(c->part); f(c->scal); f(c->ecyc); f(c->ecyclo);
  for (int l = 0; l < kMaxLevels; ++l) {
    f(c->lev[l].st); f(c->lev[l].x); f(c->lev[l].b); f(c->lev[l].t); f(c->lev[l].sth);
  }
  if (c->hscal) cudaFreeHost(c->hscal);
  for (auto& r : c->pending) {
    cudaEventDestroy(r.a);
    cudaEventDestroy(r.b);
  }
  for (auto e : c->event_pool) cudaEventDestroy(e);
  for (auto& g : c->cg_graph)
    if (g) cudaGraphExecDestroy(g);
}

bool valid_ptr(const void* p) { return p != nullptr; }

cudaEvent_t take_event(homo_ctx* c) {
  if (!c->event_pool.empty()) {
    cudaEvent_t e = c->event_pool.back();
    c->event_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
  return e;
}

// Accumulate the recorded event pairs; the stream must have been synchronised.
void prof_flush(homo_ctx* c) {
  for (auto& r : c->pending) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, r.a, r.b) == cudaSuccess) {
      c->prof_ms[r.kc] += ms;
    }
    c->event_pool.push_back(r.a);
    c->event_pool.push_back(r.b);
  }
  c->pending.clear();
}

// Counts the kernels of one launcher call and, when profiling, brackets them with events.
struct Prof {
  homo_ctx* c;
  int kc;
  cudaEvent_t a = nullptr;
  Prof(homo_ctx* ctx, int k, int nkernels) : c(ctx), kc(k) {
    c->launches += nkernels;
    if (c->prof) {
      c->prof_n[kc] += nkernels;
      if (c->pending.size() > 8192 && cudaStreamSynchronize(c->stream) == cudaSuccess) prof_flush(c);
      a = take_event(c);
      if (a) cudaEventRecord(a, c->stream);
    }
  }
  ~Prof() {
    if (!a) return;
    cudaEvent_t b = take_event(c);
    if (!b) return;
    cudaEventRecord(b, c->stream);
    c->pending.push_back({kc, a, b});
  }
};

#define KL(ctx, kc, nk, call)      \
  do {                             \
    Prof prof_(ctx, kc, nk);       \
    CK(ctx, call);                 \
  } while (0)

// Loads of a case whose norm is below this fraction of the largest case's are the
// rounding residue of a load that is zero in exact arithmetic (in-plane shear of a
// laminate, say: the double-float loads keep the 1e-16 asymmetries of K0 chi) and are set
// to zero, so the case is converged at u = 0 instead of chasing a relative tolerance on
// noise.
constexpr double kLoadResidue = 1e-12;

int ensure_loads(homo_ctx* c) {
  if (!c->density_set) return set_err(c, HOMO_ESTATE, "no density set (call homo_set_density first)");
  if (!c->loads_valid) {
    KL(c, HOMO_KC_SETUP, 1, launch_loads(c, c->f));
    int g = 0;
    KL(c, HOMO_KC_SETUP, 1, launch_dot6(c->f, c->f, c->N, c->part, &g, c->stream));
    KL(c, HOMO_KC_SETUP, 1, launch_sum_partials(c->part, g, kCases, c->scal + S_FF, c->stream));
    CK(c, cudaMemcpyAsync(c->hscal + S_FF, c->scal + S_FF, sizeof(double) * kCases, cudaMemcpyDeviceToHost,
                          c->stream));
    CK(c, cudaStreamSynchronize(c->stream));
    prof_flush(c);
    double mx = 0.0;
    for (int k = 0; k < kCases; ++k) mx = std::max(mx, c->hscal[S_FF + k]);
    for (int k = 0; k < kCases; ++k)
      if (c->hscal[S_FF + k] <= kLoadResidue * kLoadResidue * mx) {
        CK(c, cudaMemsetAsync(c->f + 3 * k * c->N, 0, sizeof(float) * 3 * c->N, c->stream));
        CK(c, cudaMemsetAsync(c->flo + 3 * k * c->N, 0, sizeof(float) * 3 * c->N, c->stream));
      }
    c->loads_valid = true;
  }
  return HOMO_OK;
}

// Upper end of the spectrum of D^-1 K on every smoothed level (Chebyshev smoother): the
// element bound on the finest level, 12 power-iteration steps times 1.15 on coarse levels.
int estimate_spectra(homo_ctx* c) {
  cudaStream_t s = c->stream;
  c->lam[0] = element_jacobi_bound(c->ke);
  for (int l = 1; l + 1 < c->nlev; ++l) {
    Level& L = c->lev[l];
    float* x = L.x;
    float* y = L.t;
    KL(c, HOMO_KC_SETUP, 1, launch_fill_hash(x, kPlanes * L.N, 0x5eed0000u + static_cast<unsigned>(l), s));
    for (int it = 0; it < 12; ++it) {
      KL(c, HOMO_KC_SETUP, 1, launch_coarse_dinvk(L, x, y, s));
      std::swap(x, y);
    }
    // x = (D^-1 K)^12 x0, y = (D^-1 K)^11 x0
    int g = 0;
    KL(c, HOMO_KC_SETUP, 1, launch_dot6(x, x, L.N, c->part, &g, s));
    KL(c, HOMO_KC_SETUP, 1, launch_sum_partials(c->part, g, kCases, c->scal + S_OC, s));
    KL(c, HOMO_KC_SETUP, 1, launch_dot6(y, y, L.N, c->part, &g, s));
    KL(c, HOMO_KC_SETUP, 1, launch_sum_partials(c->part, g, kCases, c->scal + S_OC + 8, s));
    CK(c, cudaMemcpyAsync(c->hscal + S_OC, c->scal + S_OC, sizeof(double) * 14, cudaMemcpyDeviceToHost, s));
    CK(c, cudaStreamSynchronize(s));
    prof_flush(c);
    double nx = 0, ny = 0;
    for (int k = 0; k < kCases; ++k) {
      nx += c->hscal[S_OC + k];
      ny += c->hscal[S_OC + 8 + k];
    }
    if (!(ny > 0) || !std::isfinite(nx)) return set_err(c, HOMO_EDIVERGED, "coarse spectrum estimate failed");
    c->lam[l] = 1.15 * std::sqrt(nx / ny);
  }
  return HOMO_OK;
}

int ensure_hierarchy(homo_ctx* c) {
  RET(ensure_loads(c));
  if (c->hier_valid) return HOMO_OK;
  if (c->nlev == 1) {
    KL(c, HOMO_KC_SETUP, 1, launch_fine_stencil(c, c->lev[0]));
  } else {
    KL(c, HOMO_KC_SETUP, 1, launch_level1_assemble(c, c->lev[1]));
    // the fine CG vectors z and q are free while the hierarchy is built (18 N floats each;
    // the intermediates of level 1 need 243 N / 16 and 243 N / 32)
    for (int l = 1; l + 1 < c->nlev; ++l)
      KL(c, HOMO_KC_SETUP, 3, launch_galerkin(c->lev[l], c->lev[l + 1], c->z, c->q, c->stream));
  }
  KL(c, HOMO_KC_SETUP, 3, launch_coarsest_setup(c));
  if (c->opts.smoother == HOMO_SMOOTH_CHEBYSHEV)   // captured Chebyshev coefficients go stale
    for (auto& gr : c->cg_graph)
      if (gr) {
        cudaGraphExecDestroy(gr);
        gr = nullptr;
      }
  for (int l = 1; l + 1 < c->nlev; ++l)
    if (c->lev[l].sth) KL(c, HOMO_KC_SETUP, 1, launch_stencil_bf16(c->lev[l], c->stream));
  if (c->opts.smoother == HOMO_SMOOTH_CHEBYSHEV) RET(estimate_spectra(c));
  c->hier_valid = true;
  return HOMO_OK;
}

// One 8-colour sweep. first: the sweep starts from x = 0 (x need not be cleared; only
// valid with colours in increasing order).
// fmean (finest level only): plane means subtracted from f, or null.
int smooth_level(homo_ctx* c, int l, bool reverse, const float* f, float* x, bool first = false,
                 const double* fmean = nullptr) {
  const int fz = first && !reverse ? 1 : 0;
  for (int k = 0; k < 8; ++k) {
    const int col = reverse ? 7 - k : k;
    if (l == 0) KL(c, HOMO_KC_FINE_GS, 1, launch_fine_gs(c, col, f, x, fz, fmean));
    else if (c->lev[l].n <= c->gs_split_n)
      KL(c, HOMO_KC_COARSE_GS, 1, launch_coarse_gs_item(c->lev[l], col, f, x, fz, c->stream));
    else KL(c, HOMO_KC_COARSE_GS, 1, launch_coarse_gs(c->lev[l], col, f, x, fz, c->stream));
  }
  return HOMO_OK;
}

// sweeps 8-colour sweeps on level l; first: the first sweep starts from x = 0. A small
// coarse level runs them all as one launch of per-case clusters (its displacement resident
// in shared memory up to gs_res_n cells per axis, read through L2 up to gs_fuse_n), larger
// levels one launch per colour (the per-colour launches of the small levels are mostly
// launch and load latency).
int smooth_level_sweeps(homo_ctx* c, int l, bool reverse, const float* f, float* x, int sweeps,
                        bool first = false) {
  if (sweeps < 1) return HOMO_OK;
  if (l >= 1 && c->gs_resident > 0 && c->lev[l].n <= c->gs_res_n && coarse_resident_ok(c->lev[l], c->gs_resident)) {
    KL(c, HOMO_KC_COARSE_GS, 1,
       launch_coarse_gs_resident(c->lev[l], sweeps, reverse ? 1 : 0, first && !reverse ? 1 : 0, f, x,
                                 c->gs_resident, c->stream));
    return HOMO_OK;
  }
  if (l >= 1 && c->gs_cluster > 0 && c->lev[l].n <= c->gs_fuse_n) {
    KL(c, HOMO_KC_COARSE_GS, 1,
       launch_coarse_gs_sweeps(c->lev[l], sweeps, reverse ? 1 : 0, first && !reverse ? 1 : 0, f, x,
                               c->gs_cluster, c->stream));
    return HOMO_OK;
  }
  for (int k = 0; k < sweeps; ++k) RET(smooth_level(c, l, reverse, f, x, first && k == 0));
  return HOMO_OK;
}

// Smoothing sweeps before (and after) the coarse correction on coarse level l >= 1.
int level_sweeps(const homo_ctx* c, int l) {
  int s = c->opts.coarse_sweeps;
  for (int k = 1; k < l; ++k) s = std::min(HOMO_MAX_LEVEL_SWEEPS, s * c->opts.sweep_growth);
  return s;
}

// Chebyshev iteration coefficients on [lam/10, lam] (three-term recurrence): step 0
// x1 = x0 + (1/theta) D^-1 r0; step k >= 1 x_(k+1) = x_k + ca_k (x_k - x_(k-1)) + cb_k D^-1 r_k.
struct ChebCoef {
  float c0;
  float ca[4], cb[4];
};

ChebCoef cheb_coef(double lam, int deg) {
  ChebCoef k{};
  const double hi = lam, lo = lam / 10.0;
  const double theta = 0.5 * (hi + lo), delta = 0.5 * (hi - lo), sigma = theta / delta;
  double rho_prev = 1.0 / sigma;
  k.c0 = static_cast<float>(1.0 / theta);
  for (int s = 1; s < deg && s < 4; ++s) {
    const double rho = 1.0 / (2.0 * sigma - rho_prev);
    k.ca[s] = static_cast<float>(rho * rho_prev);
    k.cb[s] = static_cast<float>(2.0 * rho / delta);
    rho_prev = rho;
  }
  return k;
}

// One Chebyshev sweep of degree cheb_degree on level l. cur holds x (ignored when
// from_zero), oth is free; on return cur holds the new x and oth is free. bmean (finest
// level only): plane means subtracted from b, or null.
int cheb_sweep(homo_ctx* c, int l, const float* b, const double* bmean, float*& cur, float*& oth,
               bool from_zero) {
  const int deg = c->opts.cheb_degree;
  const ChebCoef k = cheb_coef(c->lam[l], deg);
  if (l == 0) {
    if (from_zero) KL(c, HOMO_KC_FINE_CHEB, 1, launch_fine_jacobi_start(c, b, bmean, oth, k.c0));
    else KL(c, HOMO_KC_FINE_CHEB, 1, launch_fine_tiled(c, 4, cur, b, oth, nullptr, nullptr, bmean, k.c0, 0.f));
    std::swap(cur, oth);
    for (int s = 1; s < deg; ++s) {
      const int mode = (from_zero && s == 1) ? 6 : 5;
      KL(c, HOMO_KC_FINE_CHEB, 1, launch_fine_tiled(c, mode, cur, b, oth, nullptr, nullptr, bmean, k.ca[s], k.cb[s]));
      std::swap(cur, oth);
    }
  } else {
    const Level& L = c->lev[l];
    KL(c, HOMO_KC_COARSE_CHEB, 1, launch_coarse_cheb(L, b, from_zero ? nullptr : cur, oth, 0, k.c0, 0.f, c->stream));
    std::swap(cur, oth);
    for (int s = 1; s < deg; ++s) {
      const int mode = (from_zero && s == 1) ? 3 : 1;
      KL(c, HOMO_KC_COARSE_CHEB, 1, launch_coarse_cheb(L, b, cur, oth, mode, k.ca[s], k.cb[s], c->stream));
      std::swap(cur, oth);
    }
  }
  return HOMO_OK;
}

// V-cycle with Chebyshev smoothing (same polynomial before and after the coarse
// correction, so M is symmetric); two buffers per level alternate as iterates.
int vcycle_cheb(homo_ctx* c, const float* r, float* z, const double* rmean) {
  cudaStream_t s = c->stream;
  const int pre = c->opts.pre_sweeps, post = c->opts.post_sweeps;
  const int L = c->nlev - 1;
  float* cur[kMaxLevels];
  float* oth[kMaxLevels];
  cur[0] = z;
  oth[0] = c->q;
  for (int k = 0; k < pre; ++k) RET(cheb_sweep(c, 0, r, rmean, cur[0], oth[0], k == 0));
  KL(c, HOMO_KC_FINE_RESIDUAL, 1, launch_fine_residual(c, r, cur[0], nullptr, oth[0], nullptr, nullptr, rmean));
  KL(c, HOMO_KC_TRANSFER, 1, launch_restrict(c->n, oth[0], c->lev[1].b, s));
  for (int l = 1; l < L; ++l) {
    Level& lv = c->lev[l];
    cur[l] = lv.x;
    oth[l] = lv.t;
    for (int k = 0; k < level_sweeps(c, l); ++k) RET(cheb_sweep(c, l, lv.b, nullptr, cur[l], oth[l], k == 0));
    KL(c, HOMO_KC_COARSE_RESIDUAL, 1, launch_coarse_residual(lv, lv.b, cur[l], oth[l], s));
    KL(c, HOMO_KC_TRANSFER, 1, launch_restrict(lv.n, oth[l], c->lev[l + 1].b, s));
  }
  KL(c, HOMO_KC_COARSEST, 1, launch_coarsest_apply(c, c->lev[L].b, c->lev[L].x));
  cur[L] = c->lev[L].x;
  for (int l = L - 1; l >= 1; --l) {
    Level& lv = c->lev[l];
    KL(c, HOMO_KC_TRANSFER, 1, launch_prolong_add(lv.n, cur[l + 1], cur[l], 0, s));
    for (int k = 0; k < level_sweeps(c, l); ++k) RET(cheb_sweep(c, l, lv.b, nullptr, cur[l], oth[l], false));
  }
  KL(c, HOMO_KC_TRANSFER, 1, launch_prolong_add(c->n, cur[1], cur[0], 0, s));
  for (int k = 0; k < post; ++k) RET(cheb_sweep(c, 0, r, rmean, cur[0], oth[0], false));
  if (cur[0] != z)
    CK(c, cudaMemcpyAsync(z, cur[0], sizeof(float) * kPlanes * c->N, cudaMemcpyDeviceToDevice, s));
  return HOMO_OK;
}

// z = M (r - rmean): one symmetric V-cycle (Alg. 1) from a zero initial guess; with
// Gauss-Seidel the post-smoother visits the colours in reverse order so M is symmetric.
// rmean: the 18 plane means of r (the rigid-translation part, outside the range of K),
// or null.
int vcycle(homo_ctx* c, const float* r, float* z, const double* rmean = nullptr) {
  cudaStream_t s = c->stream;
  if (c->nlev == 1) {   // the centred pseudo-inverse ignores the plane means
    KL(c, HOMO_KC_COARSEST, 1, launch_coarsest_apply(c, r, z));
    return HOMO_OK;
  }
  if (c->opts.smoother == HOMO_SMOOTH_CHEBYSHEV) return vcycle_cheb(c, r, z, rmean);
  const int pre = c->opts.pre_sweeps, post = c->opts.post_sweeps;
  if (pre == 0) CK(c, cudaMemsetAsync(z, 0, sizeof(float) * kPlanes * c->N, s));
  for (int k = 0; k < pre; ++k) RET(smooth_level(c, 0, false, r, z, k == 0, rmean));
  KL(c, HOMO_KC_FINE_RESIDUAL, 1, launch_fine_residual(c, r, z, nullptr, c->q, nullptr, nullptr, rmean));
  KL(c, HOMO_KC_TRANSFER, 1, launch_restrict(c->n, c->q, c->lev[1].b, s));
  const int L = c->nlev - 1;
  for (int l = 1; l < L; ++l) {
    Level& lv = c->lev[l];
    RET(smooth_level_sweeps(c, l, false, lv.b, lv.x, level_sweeps(c, l), true));
    KL(c, HOMO_KC_COARSE_RESIDUAL, 1, launch_coarse_residual(lv, lv.b, lv.x, lv.t, s));
    KL(c, HOMO_KC_TRANSFER, 1, launch_restrict(lv.n, lv.t, c->lev[l + 1].b, s));
  }
  KL(c, HOMO_KC_COARSEST, 1, launch_coarsest_apply(c, c->lev[L].b, c->lev[L].x));
  for (int l = L - 1; l >= 1; --l) {
    Level& lv = c->lev[l];
    KL(c, HOMO_KC_TRANSFER, 1, launch_prolong_add(lv.n, c->lev[l + 1].x, lv.x, 0, s));
    RET(smooth_level_sweeps(c, l, true, lv.b, lv.x, level_sweeps(c, l)));
  }
  KL(c, HOMO_KC_TRANSFER, 1, launch_prolong_add(c->n, c->lev[1].x, z, 0, s));
  for (int k = 0; k < post; ++k) RET(smooth_level(c, 0, true, r, z, false, rmean));
  return HOMO_OK;
}

int sync_read(homo_ctx* c, int slot, int count) {
  CK(c, cudaMemcpyAsync(c->hscal + slot, c->scal + slot, sizeof(double) * count,
                        cudaMemcpyDeviceToHost, c->stream));
  CK(c, cudaStreamSynchronize(c->stream));
  prof_flush(c);
  return HOMO_OK;
}

// Copy count slots from the device to the pinned host mirror (no synchronisation).
int enq_read(homo_ctx* c, int slot, int count) {
  CK(c, cudaMemcpyAsync(c->hscal + slot, c->scal + slot, sizeof(double) * count,
                        cudaMemcpyDeviceToHost, c->stream));
  return HOMO_OK;
}

// r = f - K (u + ulo); ||r_c - mean||^2 into S_RR, the plane means (the rigid
// translations, outside the range of K) into S_RMEAN, active flags; enqueues the copy of
// S_RR to the host (no synchronisation).
// exact: double-float arithmetic throughout (residuals to ~1e-12 of the terms); otherwise
// FP32 difference form from both parts of u (accurate to ~1e-7 of sum_d |A_d| |du_d|,
// several times faster).
int enq_true_residual(homo_ctx* c, double tol, bool exact) {
  int g = 0;
  if (exact)
    KL(c, HOMO_KC_TRUE_RESIDUAL, 1, launch_fine_residual(c, c->f, c->u, c->ulo, c->r, c->part, &g, nullptr));
  else
    KL(c, HOMO_KC_TRUE_RESIDUAL, 1,
       launch_fine_tiled(c, 2, c->u, c->f, c->r, c->part, &g, nullptr, 0.f, 0.f, c->ulo));
  KL(c, HOMO_KC_CG_VECTOR, 1, launch_sum_partials(c->part, g, kCases + kPlanes, c->scal + S_RR, c->stream));
  KL(c, HOMO_KC_CG_VECTOR, 1, launch_cg_active(c->scal, tol, c->N, c->stream));
  return enq_read(c, S_RR, 6);
}

int true_residual(homo_ctx* c, double tol, bool exact) {
  RET(enq_true_residual(c, tol, exact));
  CK(c, cudaStreamSynchronize(c->stream));
  prof_flush(c);
  return HOMO_OK;
}

// At tolerances from this one up, a solve starts from the FP32 residual: its error (below
// 1e-6 of ||f|| at 64^3, growing about like n^(1/2)) is independent of the CG error and
// adds to it in quadrature, and the exact residual that closes every cycle catches the
// rare overshoot. Every cycle is closed, and every result certified, by the exact one.
constexpr double kFastStartTol = 1e-5;

void record_history(homo_ctx* c) {
  for (int k = 0; k < kCases; ++k) {
    const double ff = c->hscal[S_FF + k], rr = c->hscal[S_RR + k];
    c->history.push_back(ff > 0.0 ? std::sqrt(rr / ff) : 0.0);
  }
}

int precondition_and_direction(homo_ctx* c, int first) {
  int g = 0;
  RET(vcycle(c, c->r, c->z, c->scal + S_RMEAN));
  KL(c, HOMO_KC_CG_VECTOR, 1, launch_dot6_zsum(c->r, c->z, c->N, c->scal + S_RMEAN, c->part, &g, c->stream));
  KL(c, HOMO_KC_CG_VECTOR, 1, launch_sum_partials(c->part, g, kCases + kPlanes, c->scal + S_RZ, c->stream));
  KL(c, HOMO_KC_CG_VECTOR, 1, launch_cg_beta(c->scal, first, c->stream));
  KL(c, HOMO_KC_CG_VECTOR, 1, launch_cg_update_p(c->pv, c->z, c->scal, c->N, c->stream));
  return HOMO_OK;
}

// ---------------------------------------------------------------- CG solve
// Restarted CG (mixed-precision iterative refinement, u kept in double-float): a cycle runs
// on the FP32 recursive residual and accumulates its correction in double-float (ecyc +
// ecyclo), folded into u once per cycle. The residual's plane means (rigid translations,
// which K cannot produce and the V-cycle would amplify) are tracked and subtracted by every
// consumer. A cycle ends when every case meets the inner tolerance, has reduced its
// residual by kCycleDrop, or starts to grow; the next cycle starts from the exact true
// residual, which also decides convergence.
//
// The solve is a state machine: every step enqueues work on the context's stream and asks
// for one synchronisation before the next step reads the copied residual norms. A single
// solve is a batch of one; a batch advances many contexts in lockstep, all their streams
// running concurrently between synchronisations.
constexpr double kCycleDrop = 1e-5;
constexpr int kMaxCycles = 24;

struct SolveState {
  homo_ctx* c = nullptr;
  double rel_tol = 0.0, inner_tol = 0.0;
  int max_iters = 0;
  int its[kCases] = {0, 0, 0, 0, 0, 0};
  int total = 0, cycle = 0;
  bool diverged = false, accurate_last = false, first = true;
  double rr0[kCases] = {}, rrmin[kCases] = {};
  enum Phase { kInit, kAfterInit, kAfterIter, kAfterCycleRes, kAfterFinalRes, kDone } phase = kInit;
  int status = HOMO_OK;
};

bool any_active(SolveState& s, double tol) {
  homo_ctx* c = s.c;
  bool a = false;
  for (int k = 0; k < kCases; ++k) {
    const double rr = c->hscal[S_RR + k];
    if (!std::isfinite(rr)) s.diverged = true;
    if (c->hscal[S_FF + k] > 0.0 && rr > tol * tol * c->hscal[S_FF + k]) a = true;
  }
  return a;
}

bool use_graphs(const homo_ctx* c) { return c->opts.graphs && c->stream && !c->prof; }

void drop_graphs(homo_ctx* c) {
  for (auto& g : c->cg_graph)
    if (g) {
      cudaGraphExecDestroy(g);
      g = nullptr;
    }
}

// One CG iteration: direction from the preconditioned residual, product, step, new residual
// norms, copy of the norms to the host.
int enq_iteration(homo_ctx* c, int first, double inner_tol) {
  int g = 0;
  RET(precondition_and_direction(c, first));
  KL(c, HOMO_KC_FINE_MATVEC, 1, launch_fine_apply(c, c->pv, c->q, c->part, &g));
  KL(c, HOMO_KC_CG_VECTOR, 1, launch_sum_partials(c->part, g, kCases + kPlanes, c->scal + S_PQ, c->stream));
  KL(c, HOMO_KC_CG_VECTOR, 1, launch_cg_alpha(c->scal, c->stream));
  KL(c, HOMO_KC_CG_VECTOR, 1,
     launch_cg_update_er(c->ecyc, c->ecyclo, c->r, c->pv, c->q, c->scal, c->N, c->part, &g, c->stream));
  KL(c, HOMO_KC_CG_VECTOR, 1, launch_sum_partials(c->part, g, kCases + kPlanes, c->scal + S_RR, c->stream));
  KL(c, HOMO_KC_CG_VECTOR, 1, launch_cg_active(c->scal, inner_tol, c->N, c->stream));
  return enq_read(c, S_RR, 6);
}

// The same, replayed from a captured graph when the context asks for graphs. Kernel
// arguments are captured by value: pointers, sizes and the inner tolerance (recaptured
// when it changes); the smoother's Chebyshev coefficients make the graphs stale whenever
// the hierarchy is rebuilt (dropped in ensure_hierarchy).
int run_iteration(homo_ctx* c, int first, double inner_tol) {
  if (!use_graphs(c)) return enq_iteration(c, first, inner_tol);
  if (c->cg_graph[first] && c->cg_graph_tol != inner_tol) drop_graphs(c);
  if (!c->cg_graph[first]) {
    const long long l0 = c->launches;
    CK(c, cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal));
    const int rc = enq_iteration(c, first, inner_tol);
    cudaGraph_t graph = nullptr;
    const cudaError_t e = cudaStreamEndCapture(c->stream, &graph);
    if (rc != HOMO_OK) {
      if (graph) cudaGraphDestroy(graph);
      return rc;
    }
    if (e != cudaSuccess) return cuda_err(c, e, "CG iteration graph capture");
    const cudaError_t ei = cudaGraphInstantiate(&c->cg_graph[first], graph, 0);
    cudaGraphDestroy(graph);
    if (ei != cudaSuccess) {
      c->cg_graph[first] = nullptr;
      return cuda_err(c, ei, "CG iteration graph instantiation");
    }
    c->cg_graph_launches[first] = c->launches - l0;
    c->cg_graph_tol = inner_tol;
    c->launches = l0;
  }
  CK(c, cudaGraphLaunch(c->cg_graph[first], c->stream));
  c->launches += c->cg_graph_launches[first];
  return HOMO_OK;
}

void finish_solve(SolveState& s, int* iters_out, double* relres_out) {
  homo_ctx* c = s.c;
  c->solved = true;
  bool conv = true;
  for (int k = 0; k < kCases; ++k) {
    const double ff = c->hscal[S_FF + k], rr = c->hscal[S_RR + k];
    const double rel = ff > 0.0 ? std::sqrt(rr / ff) : 0.0;
    if (!std::isfinite(rr)) s.diverged = true;
    if (ff > 0.0 && !(rel <= s.rel_tol)) conv = false;
    if (relres_out) relres_out[k] = rel;
    if (iters_out) iters_out[k] = s.its[k];
  }
  if (s.diverged) s.status = set_err(c, HOMO_EDIVERGED, "non-finite residual in CG");
  else if (!conv) s.status = set_err(c, HOMO_ENOCONV, "relative residual above tolerance after max_iters");
  s.phase = SolveState::kDone;
}

// Close the solve: confirm with the exact residual unless the last cycle did.
// Returns true when work was enqueued (a synchronisation is needed).
bool begin_finish(SolveState& s, int* iters_out, double* relres_out) {
  if (!s.accurate_last && !s.diverged) {
    s.status = enq_true_residual(s.c, s.rel_tol, true);
    if (s.status != HOMO_OK) {
      s.phase = SolveState::kDone;
      return false;
    }
    s.phase = SolveState::kAfterFinalRes;
    return true;
  }
  finish_solve(s, iters_out, relres_out);
  return false;
}

bool begin_iteration(SolveState& s, int* iters_out, double* relres_out);

int enq_fold(homo_ctx* c) {
  KL(c, HOMO_KC_CG_VECTOR, 1, launch_fold(c->u, c->ulo, c->ecyc, c->ecyclo, kPlanes * c->N, c->stream));
  return HOMO_OK;
}

// End a cycle: fold the correction into u and recompute the exact residual.
bool end_cycle(SolveState& s, int* iters_out, double* relres_out) {
  homo_ctx* c = s.c;
  const int rc = enq_fold(c);
  if (rc != HOMO_OK) {
    s.status = rc;
    s.phase = SolveState::kDone;
    return false;
  }
  if (s.diverged) return begin_finish(s, iters_out, relres_out);
  s.status = enq_true_residual(c, s.rel_tol, true);   // recursive and true residual can drift apart
  if (s.status != HOMO_OK) {
    s.phase = SolveState::kDone;
    return false;
  }
  s.phase = SolveState::kAfterCycleRes;
  return true;
}

// Start a cycle, or finish when nothing is left to do.
bool begin_cycle(SolveState& s, int* iters_out, double* relres_out) {
  if (s.cycle >= kMaxCycles || s.diverged || !any_active(s, s.rel_tol) || s.total >= s.max_iters)
    return begin_finish(s, iters_out, relres_out);
  for (int k = 0; k < kCases; ++k) s.rr0[k] = s.rrmin[k] = s.c->hscal[S_RR + k];
  s.first = true;
  return begin_iteration(s, iters_out, relres_out);
}

bool begin_iteration(SolveState& s, int* iters_out, double* relres_out) {
  homo_ctx* c = s.c;
  if (s.total >= s.max_iters) return end_cycle(s, iters_out, relres_out);
  ++s.total;
  for (int k = 0; k < kCases; ++k)
    if (c->hscal[S_FF + k] > 0.0 && c->hscal[S_RR + k] > s.inner_tol * s.inner_tol * c->hscal[S_FF + k]) ++s.its[k];
  s.status = run_iteration(c, s.first ? 1 : 0, s.inner_tol);
  if (s.status != HOMO_OK) {
    s.phase = SolveState::kDone;
    return false;
  }
  s.first = false;
  s.phase = SolveState::kAfterIter;
  return true;
}

// Advance after the previous step's work has completed. Returns true when new work was
// enqueued and a synchronisation is needed before the next call.
bool advance(SolveState& s, int warm_start, int* iters_out, double* relres_out) {
  homo_ctx* c = s.c;
  switch (s.phase) {
    case SolveState::kInit: {
      s.status = ensure_hierarchy(c);
      if (s.status != HOMO_OK) break;
      const size_t V = kPlanes * c->N;
      auto enq = [&]() -> int {
        if (!warm_start) {
          CK(c, cudaMemsetAsync(c->u, 0, sizeof(float) * V, c->stream));
          CK(c, cudaMemsetAsync(c->ulo, 0, sizeof(float) * V, c->stream));
        }
        int g = 0;
        KL(c, HOMO_KC_CG_VECTOR, 1, launch_dot6(c->f, c->f, c->N, c->part, &g, c->stream));
        KL(c, HOMO_KC_CG_VECTOR, 1, launch_sum_partials(c->part, g, kCases, c->scal + S_FF, c->stream));
        RET(enq_true_residual(c, s.inner_tol, s.rel_tol < kFastStartTol));
        RET(enq_read(c, S_FF, 6));
        // the coarsest factorisation reports a failed pivot in an int next to the OC slots
        RET(enq_read(c, S_OC + 63, 1));
        CK(c, cudaMemsetAsync(c->ecyc, 0, sizeof(float) * V, c->stream));
        CK(c, cudaMemsetAsync(c->ecyclo, 0, sizeof(float) * V, c->stream));
        return HOMO_OK;
      };
      s.status = enq();
      if (s.status != HOMO_OK) break;
      s.phase = SolveState::kAfterInit;
      return true;
    }
    case SolveState::kAfterInit: {
      int piv_fail = 0;
      std::memcpy(&piv_fail, c->hscal + S_OC + 63, sizeof(int));
      if (piv_fail) {
        s.status = set_err(c, HOMO_EDIVERGED, "coarsest operator is not positive definite");
        break;
      }
      c->history.clear();
      record_history(c);
      return begin_cycle(s, iters_out, relres_out);
    }
    case SolveState::kAfterIter: {
      record_history(c);
      if (!any_active(s, s.inner_tol) || s.diverged) return end_cycle(s, iters_out, relres_out);
      bool cycle_done = true, blowup = false;
      for (int k = 0; k < kCases; ++k) {
        const double rr = c->hscal[S_RR + k], ff = c->hscal[S_FF + k];
        const bool act = ff > 0.0 && rr > s.inner_tol * s.inner_tol * ff;
        if (act && rr > kCycleDrop * kCycleDrop * s.rr0[k]) cycle_done = false;
        if (rr > 1e4 * s.rrmin[k]) blowup = true;
        s.rrmin[k] = std::min(s.rrmin[k], rr);
      }
      if (cycle_done || blowup) return end_cycle(s, iters_out, relres_out);
      return begin_iteration(s, iters_out, relres_out);
    }
    case SolveState::kAfterCycleRes:
      s.accurate_last = true;
      record_history(c);
      ++s.cycle;
      return begin_cycle(s, iters_out, relres_out);
    case SolveState::kAfterFinalRes:
      record_history(c);
      finish_solve(s, iters_out, relres_out);
      return false;
    case SolveState::kDone:
      return false;
  }
  s.phase = SolveState::kDone;   // an error ended this solve
  return false;
}

// Lockstep driver: every context advances by one step, then every context with pending
// work is synchronised (their streams ran concurrently), until all are done. Per-context
// status in status[i]; the return value is HOMO_OK unless an argument is invalid.
int solve_batch(homo_ctx* const* ctxs, int count, double rel_tol, int max_iters, int warm_start,
                int* iters_out, double* relres_out, int* status) {
  if (!(rel_tol > 0.0) || max_iters < 1) {
    for (int i = 0; i < count; ++i) set_err(ctxs[i], HOMO_EINVAL, "rel_tol > 0 and max_iters >= 1 required");
    return HOMO_EINVAL;
  }
  std::vector<SolveState> st(count);
  // cycles aim slightly below the tolerance on the recursive residual; with the correction
  // kept in double-float the exact check that closes a cycle agrees with it to a few
  // digits, so it normally passes without another cycle
  for (int i = 0; i < count; ++i) {
    st[i].c = ctxs[i];
    st[i].rel_tol = rel_tol;
    st[i].inner_tol = 0.9 * rel_tol;
    st[i].max_iters = max_iters;
  }
  std::vector<char> pending(count, 0);
  for (;;) {
    bool any = false;
    for (int i = 0; i < count; ++i) {
      if (st[i].phase == SolveState::kDone) continue;
      pending[i] = advance(st[i], warm_start, iters_out ? iters_out + kCases * i : nullptr,
                           relres_out ? relres_out + kCases * i : nullptr) ? 1 : 0;
      any = any || pending[i];
    }
    if (!any) break;
    for (int i = 0; i < count; ++i) {
      if (!pending[i]) continue;
      const cudaError_t e = cudaStreamSynchronize(ctxs[i]->stream);
      if (e != cudaSuccess) {
        st[i].status = cuda_err(ctxs[i], e, "solve synchronisation");
        st[i].phase = SolveState::kDone;
      }
      prof_flush(ctxs[i]);
    }
  }
  for (int i = 0; i < count; ++i) status[i] = st[i].status;
  return HOMO_OK;
}

}  // namespace

namespace homo {
// Message returned by homo_last_error(NULL) on this thread (context-free entry points).
void set_thread_error(const std::string& msg) { g_create_err = msg; }
}  // namespace homo

extern "C" {

int homo_version(void) { return 100; }

const char* homo_status_string(int status) {
  switch (status) {
    case HOMO_OK: return "ok";
    case HOMO_EINVAL: return "invalid argument";
    case HOMO_ENOMEM: return "out of memory";
    case HOMO_ECUDA: return "CUDA error";
    case HOMO_ENOCONV: return "not converged within the iteration limit";
    case HOMO_EDIVERGED: return "diverged (non-finite residual)";
    case HOMO_ESTATE: return "call out of order";
    default: return "unknown status";
  }
}

const char* homo_last_error(const homo_ctx* ctx) {
  return ctx ? ctx->err.c_str() : g_create_err.c_str();
}

int homo_element_matrix(double nu, double Ke[576]) {
  if (!Ke || !(nu > -1.0 && nu < 0.5)) return HOMO_EINVAL;
  KeParam ke;
  LoadParam ld;
  ChiParam chi;
  build_element_matrix(nu, ke, ld, chi);
  for (int i = 0; i < 576; ++i) Ke[i] = ke.k[i];
  return HOMO_OK;
}

int homo_element_jacobi_bound(double nu, double* out) {
  if (!out || !(nu > -1.0 && nu < 0.5)) return HOMO_EINVAL;
  KeParam ke;
  LoadParam ld;
  ChiParam chi;
  build_element_matrix(nu, ke, ld, chi);
  *out = element_jacobi_bound(ke);
  return HOMO_OK;
}

int homo_create(homo_ctx** out, int n, double E0, double nu, double p, double Emin,
                const homo_opts* opts) {
  g_create_err.clear();
  if (!out) return set_err(nullptr, HOMO_EINVAL, "out is NULL");
  *out = nullptr;
  if (n < 4 || n > 1024) return set_err(nullptr, HOMO_EINVAL, "n must be in [4, 1024]");
  if (!(E0 > 0) || !(nu > -1.0 && nu < 0.5) || !(p >= 1.0) || !(Emin >= 0.0 && Emin < E0))
    return set_err(nullptr, HOMO_EINVAL, "material parameters out of range");
  homo_opts o{};
  o.min_coarse = 4;
  o.max_levels = 0;
  o.pre_sweeps = 1;
  o.post_sweeps = 1;
  o.smoother = HOMO_SMOOTH_GS8;
  o.cheb_degree = 2;
  o.precision = HOMO_PRECISION_FP32;
  o.graphs = 0;
  o.coarse_sweeps = 1;
  o.sweep_growth = 3;
  if (opts) {
    if (opts->struct_size != static_cast<int>(sizeof(homo_opts)))
      return set_err(nullptr, HOMO_EINVAL, "homo_opts.struct_size mismatch");
    if (opts->min_coarse) o.min_coarse = opts->min_coarse;
    if (opts->max_levels) o.max_levels = opts->max_levels;
    if (opts->pre_sweeps) o.pre_sweeps = opts->pre_sweeps;
    if (opts->post_sweeps) o.post_sweeps = opts->post_sweeps;
    o.smoother = opts->smoother;
    if (opts->cheb_degree) o.cheb_degree = opts->cheb_degree;
    o.precision = opts->precision;
    o.graphs = opts->graphs;
    if (opts->coarse_sweeps) o.coarse_sweeps = opts->coarse_sweeps;
    if (opts->sweep_growth) o.sweep_growth = opts->sweep_growth;
  }
  if (o.min_coarse < 3 || o.max_levels < 0 || o.max_levels > kMaxLevels || o.pre_sweeps < 0 ||
      o.post_sweeps < 0 || o.pre_sweeps > 16 || o.post_sweeps > 16 || o.pre_sweeps != o.post_sweeps ||
      (o.smoother != HOMO_SMOOTH_GS8 && o.smoother != HOMO_SMOOTH_CHEBYSHEV) || o.cheb_degree < 2 ||
      o.cheb_degree > 4 || (o.precision != HOMO_PRECISION_FP32 && o.precision != HOMO_PRECISION_MIXED) ||
      (o.graphs != 0 && o.graphs != 1) || o.coarse_sweeps < 1 || o.coarse_sweeps > HOMO_MAX_LEVEL_SWEEPS ||
      o.sweep_growth < 1 || o.sweep_growth > 8)
    return set_err(nullptr, HOMO_EINVAL,
                   "bad homo_opts (min_coarse >= 3, pre == post sweeps <= 16, smoother 0/1, degree 2..4, "
                   "precision 0/1, graphs 0/1, coarse sweeps 1..64, sweep growth 1..8)");
  int sizes[kMaxLevels];
  int nlev = 1;
  sizes[0] = n;
  while (sizes[nlev - 1] % 2 == 0 && sizes[nlev - 1] / 2 >= o.min_coarse && nlev < kMaxLevels &&
         (o.max_levels == 0 || nlev < o.max_levels)) {
    sizes[nlev] = sizes[nlev - 1] / 2;
    ++nlev;
  }
  const int nc = sizes[nlev - 1];
  if (nc > 8)
    return set_err(nullptr, HOMO_EINVAL,
                   "coarsest level has " + std::to_string(nc) +
                       " cells per axis; at most 8 are solved directly (n = m * 2^k with m <= 8)");

  homo_ctx* c = new (std::nothrow) homo_ctx;
  if (!c) return set_err(nullptr, HOMO_ENOMEM, "host allocation failed");
  c->n = n;
  c->N = static_cast<size_t>(n) * n * n;
  c->E0 = E0; c->nu = nu; c->p = p; c->Emin = Emin;
  c->opts = o;
  c->gs_cluster = coarse_cluster_size();
  c->gs_resident = coarse_resident_size();
  c->opts.struct_size = sizeof(homo_opts);
  build_element_matrix(nu, c->ke, c->ld, c->chi);
  c->hBf.assign(8 * 576, 0.f);
  build_level1_tables(c->ke, c->hBf.data());
  c->nlev = nlev;
  c->nc = nc;
  c->mc = 3 * nc * nc * nc;

  int rc = HOMO_OK;
  const size_t N = c->N, V = kPlanes * N;
  auto A = [&](float** ptr, size_t cnt, const char* w) {
    if (rc == HOMO_OK) rc = dalloc(c, ptr, cnt, w);
  };
  A(&c->rho, N, "rho"); A(&c->E, N, "E"); A(&c->tmp, N, "tmp");
  A(&c->u, V, "u"); A(&c->ulo, V, "ulo"); A(&c->f, V, "f"); A(&c->flo, V, "f (low part)");
  A(&c->r, V, "r");
  A(&c->z, V, "z"); A(&c->pv, V, "p"); A(&c->q, V, "q"); A(&c->ecyc, V, "cycle correction");
  A(&c->ecyclo, V, "cycle correction (low)");
  for (int l = 0; l < nlev; ++l) {
    Level& L = c->lev[l];
    L.n = sizes[l];
    L.N = static_cast<size_t>(L.n) * L.n * L.n;
    L.colour_blocked = (L.n % 2 == 0);
    if (l >= 1 || nlev == 1) A(&L.st, kStencil * L.N, "stencil");
    if (o.precision == HOMO_PRECISION_MIXED && l >= 1 && l + 1 < nlev && rc == HOMO_OK)
      rc = dalloc(c, &L.sth, kStencil * L.N, "stencil (bf16)");
    if (l >= 1) {
      A(&L.x, kPlanes * L.N, "level x");
      A(&L.b, kPlanes * L.N, "level b");
      if (l + 1 < nlev) A(&L.t, kPlanes * L.N, "level t");
    }
  }
  if (rc == HOMO_OK) rc = dalloc(c, &c->A, static_cast<size_t>(c->mc) * c->mc, "coarsest A");
  if (rc == HOMO_OK) rc = dalloc(c, &c->G, static_cast<size_t>(c->mc) * c->mc, "coarsest G");
  c->part_cap = std::max(static_cast<size_t>(16 * 152) * 32,
                         static_cast<size_t>(tiled_grid_blocks(n)) * (kCases + kPlanes));
  if (rc == HOMO_OK) rc = dalloc(c, &c->part, c->part_cap, "partials");
  if (rc == HOMO_OK) rc = dalloc(c, &c->scal, static_cast<size_t>(S_COUNT), "scalars");
  if (rc == HOMO_OK) {
    cudaError_t e = cudaMallocHost(reinterpret_cast<void**>(&c->hscal), sizeof(double) * S_COUNT);
    if (e != cudaSuccess) rc = cuda_err(c, e, "pinned scalars");
  }
  if (rc == HOMO_OK) {
    cudaError_t e = tiled_init();
    if (e != cudaSuccess) rc = cuda_err(c, e, "tiled kernel attributes");
  }
  if (rc == HOMO_OK) {
    cudaError_t e = cudaMemset(c->u, 0, sizeof(float) * V);
    if (e == cudaSuccess) e = cudaMemset(c->ulo, 0, sizeof(float) * V);
    if (e == cudaSuccess) e = cudaMemset(c->scal, 0, sizeof(double) * S_COUNT);
    if (e != cudaSuccess) rc = cuda_err(c, e, "initial memset");
  }
  if (rc != HOMO_OK) {
    g_create_err = c->err;
    free_all(c);
    delete c;
    return rc;
  }
  *out = c;
  return HOMO_OK;
}

int homo_destroy(homo_ctx* ctx) {
  if (!ctx) return HOMO_OK;
  if (ctx->stream) cudaStreamSynchronize(ctx->stream);
  else cudaDeviceSynchronize();
  free_all(ctx);
  delete ctx;
  return HOMO_OK;
}

int homo_set_stream(homo_ctx* ctx, void* cuda_stream) {
  if (!ctx) return HOMO_EINVAL;
  ctx->stream = static_cast<cudaStream_t>(cuda_stream);
  return HOMO_OK;
}

int homo_num_levels(const homo_ctx* ctx) { return ctx ? ctx->nlev : -HOMO_EINVAL; }

int homo_level_size(const homo_ctx* ctx, int level) {
  if (!ctx || level < 0 || level >= ctx->nlev) return -HOMO_EINVAL;
  return ctx->lev[level].n;
}

int homo_filter(homo_ctx* ctx, double radius, const float* in, float* out) {
  if (!ctx) return HOMO_EINVAL;
  if (!valid_ptr(in) || !valid_ptr(out) || in == out)
    return set_err(ctx, HOMO_EINVAL, "filter: null or aliased buffers");
  FilterParam fp;
  if (build_filter_param(radius, fp) != HOMO_OK)
    return set_err(ctx, HOMO_EINVAL, "filter radius must be in (0, 3.5]");
  KL(ctx, HOMO_KC_FILTER, 1, launch_filter(fp, ctx->n, in, out, ctx->stream));
  return HOMO_OK;
}

int homo_filter_sensitivity(homo_ctx* ctx, double radius, const float* rho, const float* dc,
                            double gamma, float* out) {
  if (!ctx) return HOMO_EINVAL;
  if (!valid_ptr(rho) || !valid_ptr(dc) || !valid_ptr(out) || out == rho || out == dc)
    return set_err(ctx, HOMO_EINVAL, "filter_sensitivity: null or aliased buffers");
  if (!(gamma > 0.0 && gamma <= 1.0)) return set_err(ctx, HOMO_EINVAL, "filter_sensitivity: gamma in (0, 1]");
  FilterParam fp;
  if (build_filter_param(radius, fp) != HOMO_OK)
    return set_err(ctx, HOMO_EINVAL, "filter radius must be in (0, 3.5]");
  KL(ctx, HOMO_KC_FILTER, 1,
     launch_sensitivity_filter(fp, ctx->n, rho, dc, static_cast<float>(gamma), out, ctx->stream));
  return HOMO_OK;
}

int homo_trig_init(homo_ctx* ctx, int nb, const double q[4], const double* weights, int nweights,
                   double volfrac, double rho_min, float* rho_out) {
  if (!ctx) return HOMO_EINVAL;
  homo_ctx* c = ctx;
  const int nt = 6 * nb;
  if (nb < 1 || nb > 3 || !q || !weights || !valid_ptr(rho_out) || nweights != nt + nt * (nt + 1) / 2)
    return set_err(c, HOMO_EINVAL, "trig_init: 1 <= nb <= 3 and one weight per member of Q_n required");
  const double qn = std::sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
  if (!(qn > 0.0) || !(rho_min >= 0.0 && rho_min < 1.0) || !(volfrac > rho_min && volfrac < 1.0))
    return set_err(c, HOMO_EINVAL, "trig_init: nonzero quaternion, 0 <= rho_min < volfrac < 1 required");
  TrigParam tp{};
  const double w = q[0] / qn, x = q[1] / qn, y = q[2] / qn, z = q[3] / qn;
  const double R[9] = {1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y),
                       2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x),
                       2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)};
  for (int i = 0; i < 9; ++i) tp.R[i] = R[i];
  tp.nb = nb;
  double wabs = 0.0;
  for (int i = 0; i < nweights; ++i) {
    tp.w[i] = weights[i];
    wabs += std::fabs(weights[i]);
  }
  // y in the fine vector z (18 N floats hold N doubles; z is free outside a solve)
  double* yv = reinterpret_cast<double*>(c->z);
  KL(c, HOMO_KC_OTHER, 1, launch_trig_basis(tp, c->n, yv, c->stream));
  const double k = 15.0, Vh = std::min(1.5 * volfrac, 1.0);
  // |y| <= sum |w|; the mean density falls from rho_min + Vh to rho_min across the bracket
  double lo = -wabs - 60.0 / k, hi = wabs + 60.0 / k;
  const double target = volfrac * static_cast<double>(c->N);
  for (int pass = 0; pass < 12 && hi - lo > 1e-13 * (1.0 + std::fabs(lo)); ++pass) {
    const double dmu = (hi - lo) / (kTrigCand - 1);
    int g = 0;
    KL(c, HOMO_KC_OTHER, 1, launch_trig_volume(yv, c->N, lo, dmu, k, Vh, rho_min, c->part, &g, c->stream));
    KL(c, HOMO_KC_OTHER, 1, launch_sum_partials(c->part, g, kTrigCand, c->scal + S_OC, c->stream));
    RET(sync_read(c, S_OC, kTrigCand));
    int last = 0;   // last candidate whose mean is still above the target
    for (int cnd = 0; cnd < kTrigCand; ++cnd)
      if (c->hscal[S_OC + cnd] > target) last = cnd;
    const double nlo = lo + last * dmu;
    hi = std::min(hi, nlo + dmu);
    lo = nlo;
  }
  KL(c, HOMO_KC_OTHER, 1, launch_trig_project(yv, c->N, 0.5 * (lo + hi), k, Vh, rho_min, rho_out, c->stream));
  CK(c, cudaStreamSynchronize(c->stream));
  return HOMO_OK;
}

int homo_symmetrize(homo_ctx* ctx, int kind, const float* in, float* out) {
  if (!ctx) return HOMO_EINVAL;
  if (!valid_ptr(in) || !valid_ptr(out)) return set_err(ctx, HOMO_EINVAL, "symmetrize: null buffer");
  SymParam sp;
  if (build_sym_param(kind, sp) != HOMO_OK) return set_err(ctx, HOMO_EINVAL, "symmetrize: unknown kind");
  KL(ctx, HOMO_KC_FILTER, 1, launch_symmetrize(sp, ctx->n, in, out, ctx->stream));
  return HOMO_OK;
}

int homo_set_density(homo_ctx* ctx, const float* rho, int on_device) {
  if (!ctx) return HOMO_EINVAL;
  if (!valid_ptr(rho)) return set_err(ctx, HOMO_EINVAL, "set_density: null rho");
  const float* src = rho;
  if (!on_device) {
    CK(ctx, cudaMemcpyAsync(ctx->rho, rho, sizeof(float) * ctx->N, cudaMemcpyHostToDevice, ctx->stream));
    src = ctx->rho;
  }
  KL(ctx, HOMO_KC_OTHER, 1, launch_simp(src, ctx->rho, ctx->E, ctx->N, static_cast<float>(ctx->p),
                      static_cast<float>(ctx->E0), static_cast<float>(ctx->Emin), ctx->stream));
  ctx->density_set = true;
  ctx->loads_valid = false;
  ctx->hier_valid = false;
  ctx->solved = false;
  return HOMO_OK;
}

int homo_solve_cases(homo_ctx* ctx, double rel_tol, int max_iters, int warm_start,
                     int iters_out[6], double relres_out[6]) {
  if (!ctx) return HOMO_EINVAL;
  homo_ctx* const list[1] = {ctx};
  int st = HOMO_OK;
  const int rc = solve_batch(list, 1, rel_tol, max_iters, warm_start, iters_out, relres_out, &st);
  return rc == HOMO_OK ? st : rc;
}

int homo_solve_batch(homo_ctx* const* ctxs, int count, double rel_tol, int max_iters, int warm_start,
                     int* iters_out, double* relres_out, int* status_out) {
  if (!ctxs || count < 1) return set_err(nullptr, HOMO_EINVAL, "solve_batch: no contexts");
  for (int i = 0; i < count; ++i) {
    if (!ctxs[i]) return set_err(nullptr, HOMO_EINVAL, "solve_batch: NULL context");
    for (int j = 0; j < i; ++j)
      if (ctxs[j] == ctxs[i]) return set_err(nullptr, HOMO_EINVAL, "solve_batch: a context appears twice");
  }
  std::vector<int> st(count, HOMO_OK);
  const int rc = solve_batch(ctxs, count, rel_tol, max_iters, warm_start, iters_out, relres_out, st.data());
  int worst = HOMO_OK;
  for (int i = 0; i < count; ++i) {
    if (status_out) status_out[i] = st[i];
    if (worst == HOMO_OK || (worst == HOMO_ENOCONV && st[i] != HOMO_OK)) worst = st[i];
  }
  return rc == HOMO_OK ? worst : rc;
}

int homo_residual(homo_ctx* ctx, int method, double relres_out[6]) {
  if (!ctx) return HOMO_EINVAL;
  if (!relres_out || (method != HOMO_RESIDUAL_FP32 && method != HOMO_RESIDUAL_DOUBLE_FLOAT))
    return set_err(ctx, HOMO_EINVAL, "residual: bad method or NULL output");
  RET(ensure_loads(ctx));
  int g = 0;
  KL(ctx, HOMO_KC_CG_VECTOR, 1, launch_dot6(ctx->f, ctx->f, ctx->N, ctx->part, &g, ctx->stream));
  KL(ctx, HOMO_KC_CG_VECTOR, 1, launch_sum_partials(ctx->part, g, kCases, ctx->scal + S_FF, ctx->stream));
  RET(true_residual(ctx, 1.0, method == HOMO_RESIDUAL_DOUBLE_FLOAT));
  RET(sync_read(ctx, S_FF, 6));
  for (int k = 0; k < kCases; ++k) {
    const double ff = ctx->hscal[S_FF + k], rr = ctx->hscal[S_RR + k];
    relres_out[k] = ff > 0.0 ? std::sqrt(rr / ff) : 0.0;
  }
  return HOMO_OK;
}

int homo_residual_field(homo_ctx* ctx, int method, const float* b, const float* u, float* out) {
  if (!ctx) return HOMO_EINVAL;
  if (!out) return set_err(ctx, HOMO_EINVAL, "residual_field: NULL output");
  if (method == HOMO_RESIDUAL_VCYCLE) {
    if (!b || !u || b == out || u == out) return set_err(ctx, HOMO_EINVAL, "residual_field: bad b/u/out");
    if (!ctx->density_set) return set_err(ctx, HOMO_ESTATE, "no density set");
    KL(ctx, HOMO_KC_FINE_RESIDUAL, 1, launch_fine_residual(ctx, b, u, nullptr, out, nullptr, nullptr, nullptr));
    CK(ctx, cudaStreamSynchronize(ctx->stream));
    prof_flush(ctx);
    return HOMO_OK;
  }
  if ((method != HOMO_RESIDUAL_FP32 && method != HOMO_RESIDUAL_DOUBLE_FLOAT) || b || u)
    return set_err(ctx, HOMO_EINVAL, "residual_field: bad method or b/u given");
  RET(ensure_loads(ctx));
  RET(true_residual(ctx, 1.0, method == HOMO_RESIDUAL_DOUBLE_FLOAT));
  CK(ctx, cudaMemcpyAsync(out, ctx->r, sizeof(float) * kPlanes * ctx->N, cudaMemcpyDeviceToDevice, ctx->stream));
  CK(ctx, cudaStreamSynchronize(ctx->stream));
  return HOMO_OK;
}

int homo_CH(homo_ctx* ctx, double CH[36]) {
  if (!ctx || !CH) return HOMO_EINVAL;
  if (!ctx->solved) return set_err(ctx, HOMO_ESTATE, "homo_CH needs a solve first");
  int g = 0;
  KL(ctx, HOMO_KC_ELEMENT, 1, launch_fine_elem(ctx, 0, nullptr, nullptr, ctx->part, &g));
  KL(ctx, HOMO_KC_CG_VECTOR, 1, launch_sum_partials(ctx->part, g, 21, ctx->scal + S_CH, ctx->stream));
  RET(sync_read(ctx, S_CH, 21));
  int idx = 0;
  const double invN = 1.0 / static_cast<double>(ctx->N);
  for (int i = 0; i < kCases; ++i)
    for (int j = i; j < kCases; ++j) {
      const double v = ctx->hscal[S_CH + idx++] * invN;
      CH[6 * i + j] = v;
      CH[6 * j + i] = v;
    }
  return HOMO_OK;
}

int homo_sensitivity(homo_ctx* ctx, const double dfdCH[36], float* dfdrho) {
  if (!ctx || !dfdCH || !dfdrho) return HOMO_EINVAL;
  if (!ctx->solved) return set_err(ctx, HOMO_ESTATE, "homo_sensitivity needs a solve first");
  KL(ctx, HOMO_KC_ELEMENT, 1, launch_fine_elem(ctx, 1, dfdCH, dfdrho, nullptr, nullptr));
  return HOMO_OK;
}

int homo_update(homo_ctx* ctx, const float* dfdrho, float* rho, double volfrac, double move,
                double damp, double rho_min, double* change_out) {
  if (!ctx) return HOMO_EINVAL;
  if (!dfdrho || !rho || static_cast<const void*>(dfdrho) == static_cast<const void*>(rho))
    return set_err(ctx, HOMO_EINVAL, "update: null or aliased buffers");
  if (!(volfrac > 0.0 && volfrac <= 1.0) || !(move > 0.0) || !(damp > 0.0) ||
      !(rho_min >= 0.0 && rho_min < 1.0))
    return set_err(ctx, HOMO_EINVAL, "update: parameters out of range");
  KL(ctx, HOMO_KC_OC, kOcKernels, launch_oc(ctx, dfdrho, rho, volfrac, move, damp, rho_min, change_out));
  return HOMO_OK;
}

int homo_objective(int kind, const double CH[36], int iteration, double param, double* f_out,
                   double dfdCH[36]) {
  if (!CH || !f_out || !dfdCH) return HOMO_EINVAL;
  auto C = [&](int i, int j) { return CH[6 * i + j]; };
  for (int i = 0; i < 36; ++i) dfdCH[i] = 0.0;
  switch (kind) {
    case HOMO_OBJ_BULK:
      *f_out = -(C(0, 0) + C(1, 1) + C(2, 2) + 2.0 * (C(0, 1) + C(0, 2) + C(1, 2))) / 9.0;
      for (int i = 0; i < 3; ++i) dfdCH[7 * i] = -1.0 / 9.0;
      dfdCH[1] = dfdCH[2] = dfdCH[8] = -2.0 / 9.0;
      return HOMO_OK;
    case HOMO_OBJ_SHEAR:
      *f_out = -(C(3, 3) + C(4, 4) + C(5, 5)) / 3.0;
      for (int i = 3; i < 6; ++i) dfdCH[7 * i] = -1.0 / 3.0;
      return HOMO_OK;
    case HOMO_OBJ_POISSON: {
      const double bl = std::pow(param, iteration);
      *f_out = C(0, 1) + C(0, 2) + C(1, 2) - bl * (C(0, 0) + C(1, 1) + C(2, 2));
      dfdCH[1] = dfdCH[2] = dfdCH[8] = 1.0;
      for (int i = 0; i < 3; ++i) dfdCH[7 * i] = -bl;
      return HOMO_OK;
    }
    case HOMO_OBJ_LOGPOISSON: {
      const double eta = 0.6, gamma = 0.5;
      const double E0 = param > 0 ? param : 1.0;
      const double tau = -1.0 / std::pow(E0, gamma);
      const double a = C(0, 1) + C(1, 2) + C(2, 0), b = C(0, 0) + C(1, 1) + C(2, 2);
      if (!(b > 0)) return HOMO_EINVAL;
      const double t = 1.0 + eta * a / b;
      *f_out = std::log(t) + tau * std::pow(b, gamma);
      const double da = eta / b / t;
      const double db = -eta * a / (b * b) / t + tau * gamma * std::pow(b, gamma - 1.0);
      dfdCH[1] = dfdCH[8] = dfdCH[12] = da;   // (0,1), (1,2), (2,0)
      for (int i = 0; i < 3; ++i) dfdCH[7 * i] = db;
      return HOMO_OK;
    }
    default:
      return HOMO_EINVAL;
  }
}

int homo_get_displacement(homo_ctx* ctx, float* u) {
  if (!ctx || !u) return HOMO_EINVAL;
  KL(ctx, HOMO_KC_OTHER, 1, launch_split_get(ctx->u, ctx->ulo, u, kPlanes * ctx->N, ctx->stream));
  return HOMO_OK;
}

int homo_set_displacement(homo_ctx* ctx, const float* u) {
  if (!ctx || !u) return HOMO_EINVAL;
  KL(ctx, HOMO_KC_OTHER, 1, launch_split_set(ctx->u, ctx->ulo, u, kPlanes * ctx->N, ctx->stream));
  ctx->solved = false;
  return HOMO_OK;
}

int homo_save_displacement(homo_ctx* ctx, float* hi, float* lo) {
  if (!ctx || !hi || !lo) return HOMO_EINVAL;
  const size_t bytes = sizeof(float) * kPlanes * ctx->N;
  CK(ctx, cudaMemcpyAsync(hi, ctx->u, bytes, cudaMemcpyDeviceToDevice, ctx->stream));
  CK(ctx, cudaMemcpyAsync(lo, ctx->ulo, bytes, cudaMemcpyDeviceToDevice, ctx->stream));
  return HOMO_OK;
}

int homo_restore_displacement(homo_ctx* ctx, const float* hi, const float* lo) {
  if (!ctx || !hi || !lo) return HOMO_EINVAL;
  const size_t bytes = sizeof(float) * kPlanes * ctx->N;
  CK(ctx, cudaMemcpyAsync(ctx->u, hi, bytes, cudaMemcpyDeviceToDevice, ctx->stream));
  CK(ctx, cudaMemcpyAsync(ctx->ulo, lo, bytes, cudaMemcpyDeviceToDevice, ctx->stream));
  ctx->solved = false;
  return HOMO_OK;
}

int homo_get_loads(homo_ctx* ctx, float* f) {
  if (!ctx || !f) return HOMO_EINVAL;
  RET(ensure_loads(ctx));
  CK(ctx, cudaMemcpyAsync(f, ctx->f, sizeof(float) * kPlanes * ctx->N, cudaMemcpyDeviceToDevice, ctx->stream));
  return HOMO_OK;
}

int homo_apply_K(homo_ctx* ctx, const float* u, float* out) {
  if (!ctx || !u || !out || u == out) return HOMO_EINVAL;
  if (!ctx->density_set) return set_err(ctx, HOMO_ESTATE, "no density set");
  KL(ctx, HOMO_KC_FINE_MATVEC, 1, launch_fine_apply(ctx, u, out, nullptr, nullptr));
  return HOMO_OK;
}

int homo_get_stencil(homo_ctx* ctx, int level, float* out) {
  if (!ctx || !out || level < 0 || level >= ctx->nlev) return HOMO_EINVAL;
  RET(ensure_hierarchy(ctx));
  if (level == 0 && !ctx->lev[0].st) {
    Level tmp = ctx->lev[0];
    if (dalloc(ctx, &tmp.st, kStencil * tmp.N, "temporary level-0 stencil") != HOMO_OK) return HOMO_ENOMEM;
    cudaError_t e = launch_fine_stencil(ctx, tmp);
    if (e == cudaSuccess) e = launch_stencil_export(tmp, out, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    cudaFree(tmp.st);
    if (e != cudaSuccess) return cuda_err(ctx, e, "level-0 stencil export");
    return HOMO_OK;
  }
  KL(ctx, HOMO_KC_OTHER, 1, launch_stencil_export(ctx->lev[level], out, ctx->stream));
  return HOMO_OK;
}

int homo_restrict(homo_ctx* ctx, int level, const float* fine, float* coarse) {
  if (!ctx || !fine || !coarse || level < 0 || level + 1 >= ctx->nlev) return HOMO_EINVAL;
  KL(ctx, HOMO_KC_TRANSFER, 1, launch_restrict(ctx->lev[level].n, fine, coarse, ctx->stream));
  return HOMO_OK;
}

int homo_prolong(homo_ctx* ctx, int level, const float* coarse, float* fine) {
  if (!ctx || !fine || !coarse || level < 0 || level + 1 >= ctx->nlev) return HOMO_EINVAL;
  KL(ctx, HOMO_KC_TRANSFER, 1, launch_prolong_add(ctx->lev[level].n, coarse, fine, 1, ctx->stream));
  return HOMO_OK;
}

int homo_set_tuning(homo_ctx* ctx, int gs_cases, int gs_block) {
  if (!ctx) return HOMO_EINVAL;
  if (!gs_variant_ok(gs_cases, gs_block)) return set_err(ctx, HOMO_EINVAL, "no such Gauss-Seidel variant");
  if (gs_cases != ctx->gs_cases || gs_block != ctx->gs_block) drop_graphs(ctx);
  ctx->gs_cases = gs_cases;
  ctx->gs_block = gs_block;
  return HOMO_OK;
}

namespace {
std::mutex g_tune_mu;
std::map<int, std::pair<int, int>> g_tune_cache;   // grid size -> (cases, block)
}  // namespace

int homo_autotune(homo_ctx* ctx, int flags, int* gs_cases, int* gs_block, double* ms) {
  if (!ctx) return HOMO_EINVAL;
  if (!ctx->density_set) return set_err(ctx, HOMO_ESTATE, "homo_autotune needs a density");
  static const int kVar[4][2] = {{3, 256}, {3, 128}, {6, 256}, {6, 128}};
  if (ms)
    for (int k = 0; k < 4; ++k) ms[k] = -1.0;
  int best = -1;
  if (!(flags & HOMO_TUNE_RETIME)) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tune_cache.find(ctx->n);
    if (it != g_tune_cache.end())
      for (int k = 0; k < 4; ++k)
        if (kVar[k][0] == it->second.first && kVar[k][1] == it->second.second) best = k;
  }
  if (best < 0) {
    // time one symmetric sweep pair (16 colour passes) of each variant on the context's
    // own moduli and loads, into the CG scratch vector z (free between solves)
    RET(ensure_loads(ctx));
    cudaEvent_t a = nullptr, b = nullptr;
    if (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess) {
      if (a) cudaEventDestroy(a);
      return set_err(ctx, HOMO_ECUDA, "homo_autotune: cudaEventCreate failed");
    }
    const int save_c = ctx->gs_cases, save_b = ctx->gs_block;
    double best_ms = 0.0;
    int rc = HOMO_OK;
    for (int k = 0; k < 4 && rc == HOMO_OK; ++k) {
      ctx->gs_cases = kVar[k][0];
      ctx->gs_block = kVar[k][1];
      rc = smooth_level(ctx, 0, false, ctx->f, ctx->z, true);            // warm-up, from zero
      if (rc != HOMO_OK) break;
      if (cudaEventRecord(a, ctx->stream) != cudaSuccess) { rc = HOMO_ECUDA; break; }
      for (int rep = 0; rep < 2 && rc == HOMO_OK; ++rep) {
        rc = smooth_level(ctx, 0, false, ctx->f, ctx->z);
        if (rc == HOMO_OK) rc = smooth_level(ctx, 0, true, ctx->f, ctx->z);
      }
      if (rc != HOMO_OK) break;
      float t = 0.f;
      if (cudaEventRecord(b, ctx->stream) != cudaSuccess || cudaEventSynchronize(b) != cudaSuccess ||
          cudaEventElapsedTime(&t, a, b) != cudaSuccess) {
        rc = HOMO_ECUDA;
        break;
      }
      if (ms) ms[k] = t / 2.0;
      if (best < 0 || t < best_ms) {
        best = k;
        best_ms = t;
      }
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    ctx->gs_cases = save_c;
    ctx->gs_block = save_b;
    if (rc != HOMO_OK) return rc == HOMO_ECUDA ? set_err(ctx, rc, "homo_autotune: timing failed") : rc;
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune_cache[ctx->n] = {kVar[best][0], kVar[best][1]};
  }
  RET(homo_set_tuning(ctx, kVar[best][0], kVar[best][1]));
  if (gs_cases) *gs_cases = kVar[best][0];
  if (gs_block) *gs_block = kVar[best][1];
  return HOMO_OK;
}

int homo_prolong_add(homo_ctx* ctx, int level, const float* coarse, float* fine) {
  if (!ctx || !fine || !coarse || level < 0 || level + 1 >= ctx->nlev) return HOMO_EINVAL;
  KL(ctx, HOMO_KC_TRANSFER, 1, launch_prolong_add(ctx->lev[level].n, coarse, fine, 0, ctx->stream));
  return HOMO_OK;
}

int homo_smooth(homo_ctx* ctx, int level, int reverse, const float* f, float* u) {
  if (!ctx || !f || !u || level < 0 || level >= ctx->nlev) return HOMO_EINVAL;
  if (ctx->lev[level].n % 2 != 0) return set_err(ctx, HOMO_EINVAL, "smoothing needs an even level size");
  RET(ensure_hierarchy(ctx));
  return smooth_level_sweeps(ctx, level, reverse != 0, f, u, 1);
}

int homo_set_coarse_smoother(homo_ctx* ctx, int resident_max_n, int cluster_max_n, int split_max_n) {
  if (!ctx) return HOMO_EINVAL;
  if (resident_max_n < 0 || resident_max_n > 1024 || cluster_max_n < 0 || cluster_max_n > 1024 ||
      split_max_n < 0 || split_max_n > 1024)
    return set_err(ctx, HOMO_EINVAL, "coarse smoother sizes must be in [0, 1024]");
  if (resident_max_n != ctx->gs_res_n || cluster_max_n != ctx->gs_fuse_n || split_max_n != ctx->gs_split_n)
    drop_graphs(ctx);
  ctx->gs_res_n = resident_max_n;
  ctx->gs_fuse_n = cluster_max_n;
  ctx->gs_split_n = split_max_n;
  return HOMO_OK;
}

namespace {
std::mutex g_coarse_tune_mu;
// (grid size, precision, level-1 sweeps, sweep growth, levels) -> (resident, cluster, split)
std::map<std::array<int, 5>, std::array<int, 3>> g_coarse_tune_cache;

// The coarse Gauss-Seidel form smooth_level_sweeps picks for level l under sizes (r, c, s):
// 0 vertex, 1 item, 2 cluster, 3 resident.
int coarse_form(const homo_ctx* ctx, int l, int r, int c, int s) {
  const homo::Level& lv = ctx->lev[l];
  if (ctx->gs_resident > 0 && lv.n <= r && homo::coarse_resident_ok(lv, ctx->gs_resident)) return 3;
  if (ctx->gs_cluster > 0 && lv.n <= c) return 2;
  return lv.n <= s ? 1 : 0;
}
}  // namespace

int homo_autotune_coarse(homo_ctx* ctx, int flags, int* resident_max_n, int* cluster_max_n, int* split_max_n,
                         double* ms) {
  if (!ctx) return HOMO_EINVAL;
  if (!ctx->density_set) return set_err(ctx, HOMO_ESTATE, "homo_autotune_coarse needs a density");
  constexpr int kForms = 4;
  static const int kSizes[kForms][3] = {{0, 0, 0}, {0, 0, 1024}, {0, 1024, 0}, {1024, 1024, 0}};
  if (ms)
    for (int k = 0; k < kMaxLevels * kForms; ++k) ms[k] = -1.0;
  const std::array<int, 5> key = {ctx->n, ctx->opts.precision, ctx->opts.coarse_sweeps, ctx->opts.sweep_growth,
                                  ctx->nlev};
  std::array<int, 3> best = {-1, -1, -1};
  if (!(flags & HOMO_TUNE_RETIME)) {
    std::lock_guard<std::mutex> lk(g_coarse_tune_mu);
    auto it = g_coarse_tune_cache.find(key);
    if (it != g_coarse_tune_cache.end()) best = it->second;
  }
  if (best[0] < 0) {
    // time each coarse level's two smoothing phases of a V-cycle (the first from zero, the
    // second in reverse colour order) in every form the level can take, on the level's own
    // stencils; the level vectors are free between solves
    RET(ensure_hierarchy(ctx));
    const int last = ctx->nlev - 1;   // the coarsest level is solved, not smoothed
    double t[kMaxLevels][kForms];
    for (auto& row : t)
      for (double& v : row) v = -1.0;
    cudaEvent_t a = nullptr, b = nullptr;
    if (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess) {
      if (a) cudaEventDestroy(a);
      return set_err(ctx, HOMO_ECUDA, "homo_autotune_coarse: cudaEventCreate failed");
    }
    const int save_r = ctx->gs_res_n, save_c = ctx->gs_fuse_n, save_s = ctx->gs_split_n;
    int rc = HOMO_OK;
    for (int l = 1; l < last && rc == HOMO_OK; ++l) {
      homo::Level& lv = ctx->lev[l];
      const int sw = level_sweeps(ctx, l);
      if (launch_fill_hash(lv.b, kPlanes * lv.N, 0x70e50000u + static_cast<unsigned>(l), ctx->stream) != cudaSuccess) {
        rc = HOMO_ECUDA;
        break;
      }
      for (int k = 0; k < kForms && rc == HOMO_OK; ++k) {
        // candidates: the per-colour item form up to 128^3, the cluster forms up to 64^3
        // (one cluster of at most 16 CTAs per load case), the resident form where it fits
        if ((k == 1 && lv.n > 128) || (k >= 2 && lv.n > 64)) continue;
        ctx->gs_res_n = kSizes[k][0];
        ctx->gs_fuse_n = kSizes[k][1];
        ctx->gs_split_n = kSizes[k][2];
        if (coarse_form(ctx, l, ctx->gs_res_n, ctx->gs_fuse_n, ctx->gs_split_n) != k) continue;
        const int reps = lv.n <= 32 ? 4 : 1;
        for (int rep = -1; rep < reps && rc == HOMO_OK; ++rep) {   // rep -1: warm-up
          if (rep == 0 && cudaEventRecord(a, ctx->stream) != cudaSuccess) rc = HOMO_ECUDA;
          if (rc == HOMO_OK) rc = smooth_level_sweeps(ctx, l, false, lv.b, lv.x, sw, true);
          if (rc == HOMO_OK) rc = smooth_level_sweeps(ctx, l, true, lv.b, lv.x, sw);
        }
        if (rc != HOMO_OK) break;
        float el = 0.f;
        if (cudaEventRecord(b, ctx->stream) != cudaSuccess || cudaEventSynchronize(b) != cudaSuccess ||
            cudaEventElapsedTime(&el, a, b) != cudaSuccess) {
          rc = HOMO_ECUDA;
          break;
        }
        t[l][k] = el / reps;
      }
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    ctx->gs_res_n = save_r;
    ctx->gs_fuse_n = save_c;
    ctx->gs_split_n = save_s;
    if (rc != HOMO_OK) return rc == HOMO_ECUDA ? set_err(ctx, rc, "homo_autotune_coarse: timing failed") : rc;
    // the sizes (each 0 or a level size) whose forms give the smallest total phase time;
    // ascending, so that of equivalent sizes the smallest is reported
    std::vector<int> cand = {0};
    for (int l = last - 1; l >= 1; --l) cand.push_back(ctx->lev[l].n);
    double best_t = -1.0;
    for (int r : cand)
      for (int c : cand)
        for (int sp : cand) {
          double tot = 0.0;
          for (int l = 1; l < last && tot >= 0.0; ++l) {
            const double v = t[l][coarse_form(ctx, l, r, c, sp)];
            tot = v < 0.0 ? -1.0 : tot + v;
          }
          if (tot >= 0.0 && (best_t < 0.0 || tot < best_t)) {
            best_t = tot;
            best = {r, c, sp};
          }
        }
    if (best[0] < 0) return set_err(ctx, HOMO_ECUDA, "homo_autotune_coarse: no form timed on every level");
    if (ms)
      for (int l = 0; l < kMaxLevels; ++l)
        for (int k = 0; k < kForms; ++k) ms[l * kForms + k] = t[l][k];
    std::lock_guard<std::mutex> lk(g_coarse_tune_mu);
    g_coarse_tune_cache[key] = best;
  }
  RET(homo_set_coarse_smoother(ctx, best[0], best[1], best[2]));
  if (resident_max_n) *resident_max_n = best[0];
  if (cluster_max_n) *cluster_max_n = best[1];
  if (split_max_n) *split_max_n = best[2];
  return HOMO_OK;
}

int homo_coarse_smoother(const homo_ctx* ctx, int* resident_max_n, int* cluster_max_n, int* split_max_n,
                         int* cluster, int* resident_cluster) {
  if (!ctx) return HOMO_EINVAL;
  if (resident_max_n) *resident_max_n = ctx->gs_res_n;
  if (cluster_max_n) *cluster_max_n = ctx->gs_fuse_n;
  if (split_max_n) *split_max_n = ctx->gs_split_n;
  if (resident_cluster) *resident_cluster = ctx->gs_resident;
  if (cluster) *cluster = ctx->gs_cluster;
  return HOMO_OK;
}

int homo_vcycle(homo_ctx* ctx, const float* r, float* z) {
  if (!ctx || !r || !z || r == z) return HOMO_EINVAL;
  RET(ensure_hierarchy(ctx));
  return vcycle(ctx, r, z);
}

int homo_profile_enable(homo_ctx* ctx, int enable) {
  if (!ctx) return HOMO_EINVAL;
  CK(ctx, cudaStreamSynchronize(ctx->stream));
  prof_flush(ctx);
  for (int k = 0; k < HOMO_KC_COUNT; ++k) {
    ctx->prof_n[k] = 0;
    ctx->prof_ms[k] = 0.0;
  }
  ctx->prof = enable != 0;
  return HOMO_OK;
}

int homo_profile_read(homo_ctx* ctx, int kc, long long* launches, double* total_ms) {
  if (!ctx || kc < 0 || kc >= HOMO_KC_COUNT) return HOMO_EINVAL;
  CK(ctx, cudaStreamSynchronize(ctx->stream));
  prof_flush(ctx);
  if (launches) *launches = ctx->prof_n[kc];
  if (total_ms) *total_ms = ctx->prof_ms[kc];
  return HOMO_OK;
}

const char* homo_kernel_class_name(int kc) {
  static const char* names[HOMO_KC_COUNT] = {
      "fine_matvec", "fine_residual", "fine_gs", "coarse_gs", "coarse_residual", "transfer", "coarsest",
      "setup", "cg_vector", "element", "filter", "oc", "other", "fine_cheb", "coarse_cheb", "true_residual"};
  return (kc >= 0 && kc < HOMO_KC_COUNT) ? names[kc] : "";
}

long long homo_launch_count(const homo_ctx* ctx) { return ctx ? ctx->launches : -1; }

int homo_residual_history(const homo_ctx* ctx, double* out, int capacity) {
  if (!ctx || capacity < 0 || (capacity > 0 && !out)) return -HOMO_EINVAL;
  const int rows = static_cast<int>(ctx->history.size() / kCases);
  const int m = std::min(rows, capacity);
  for (int i = 0; i < m * kCases; ++i) out[i] = ctx->history[i];
  return rows;
}

}  // extern "C"
