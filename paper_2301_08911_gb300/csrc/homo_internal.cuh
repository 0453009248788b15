// Internal declarations of the homo library (not part of the C ABI).
//
// Data layout on the device (voxel units, element side 1):
//   * scalar element fields (rho~, E): N = n^3 floats, x fastest.
//   * 6-case vector fields: 18 planes of N floats, plane = 3*case + comp.
//   * level l >= 1 Galerkin stencils: 243 planes of N_l floats, plane = 9*d + 3*r + c
//     (d = neighbour offset (dx+1)+3(dy+1)+9(dz+1), 3x3 block row r, column c); inside
//     a plane the vertices are grouped by Gauss-Seidel colour (Sec. 4.1 "Memory
//     layouts") when n_l is even, so one colour pass reads one contiguous 1/8 of every
//     plane; x-fastest order when n_l is odd (only possible on the coarsest level).
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>
#include <string>
#include <vector>

#include "homo.h"

namespace homo {

constexpr int kCases = 6;
constexpr int kPlanes = 18;
constexpr int kStencil = 243;
constexpr int kMaxLevels = 16;
constexpr int kRedBlock = 256;          // threads per block of every reduction kernel
constexpr int kOcPasses = 8;            // OC multiplier search passes (15 candidates each)
constexpr int kOcKernels = 4 + 3 * kOcPasses;   // kernels one OC update launches

// Element matrix of a unit-modulus voxel (side 1), row-major 24x24, dof 3j + comp.
struct KeParam {
  float k[576];
};

// Per-case nodal force of a unit-modulus element under the unit macro strain:
// fe[i][3j+comp] = (K0 chi_i)[3j+comp] (Eq. 4 with the element-relative chi of Eq. 12).
struct LoadParam {
  float fe[kCases][24];      // K0 chi_i per local dof, high part
  float fe_lo[kCases][24];   // low part (fe + fe_lo = K0 chi_i to double precision)
};

// Element-relative unit-strain displacements chi_i (Eq. 12), voxel units.
struct ChiParam {
  float chi[kCases][24];
};

// Filter weights (periodic linear cone) for up to 7^3 offsets.
struct FilterParam {
  int count;
  float inv_wsum;
  signed char off[343][3];
  float w[343];
};

// Cube symmetry group (Sec. 6.1) as signed axis permutations: the image of element
// (i0, i1, i2) has index j_k = i_perm[k], mirrored to n-1-j_k when bit k of flip is set.
struct SymParam {
  int count;
  unsigned char perm[48][3];
  unsigned char flip[48];
};

// Trigonometric initialisation (Sec. 6.2): rotation, basis size and the weights of
// Q_n (at most nb = 3: 18 + 171 weights).
constexpr int kTrigMaxT = 18;
constexpr int kTrigMaxW = kTrigMaxT + kTrigMaxT * (kTrigMaxT + 1) / 2;
struct TrigParam {
  double R[9];
  int nb;
  double w[kTrigMaxW];
};
constexpr int kTrigCand = 32;   // shift candidates per projection pass

struct Level {
  int n = 0;
  size_t N = 0;
  bool colour_blocked = false;
  float* st = nullptr;   // 243 * N (levels >= 1)
  __nv_bfloat16* sth = nullptr;   // symmetrised BF16 copy of st (mixed precision, smoothed
                                  // coarse levels), read by the coarse smoothers/residual
  float* x = nullptr;    // 18 * N (levels >= 1)
  float* b = nullptr;    // 18 * N (levels >= 1)
  float* t = nullptr;    // 18 * N residual scratch (levels >= 1)
};

// Device-side scalar slots (doubles) used by the CG driver.
// Pairs reduced by one kernel are contiguous (6 dots followed by 18 plane sums).
enum Slot : int {
  S_FF = 0,        // ||f_c||^2                  [6]
  S_RR = 6,        // ||r_c||^2                  [6]
  S_RSUM = 12,     // sum of r per plane         [18]
  S_RZ = 30,       // (r_c, z_c)                 [6]
  S_ZSUM = 36,     // sum of z per plane         [18]
  S_RZ_OLD = 54,   // previous (r_c, z_c)        [6]
  S_PQ = 60,       // (p_c, K p_c)               [6]
  S_QSUM = 66,     // sum of K p per plane       [18]
  S_ALPHA = 84,    // alpha_c                    [6]
  S_BETA = 90,     // beta_c                     [6]
  S_ACTIVE = 96,   // 1.0 while case c iterates  [6]
  S_CH = 102,      // C^H sums                   [21]
  S_OC = 128,      // OC scratch                 [64]
  S_RMEAN = 192,   // plane means of r, subtracted by every consumer of r [18]
  S_COUNT = 210
};

struct homo_ctx_impl;

}  // namespace homo

struct homo_ctx {
  int n = 0;
  size_t N = 0;
  double E0 = 1, nu = 0.3, p = 3, Emin = 1e-9;
  homo_opts opts{};
  cudaStream_t stream = nullptr;
  homo::KeParam ke{};
  homo::LoadParam ld{};
  homo::ChiParam chi{};

  float* rho = nullptr;      // filtered density, N
  float* E = nullptr;        // element moduli, N
  float* u = nullptr;        // displacement, 18N (high part)
  float* ulo = nullptr;      // displacement low part (u = u + ulo exactly), 18N
  float* ecyc = nullptr;     // correction accumulated during one CG cycle, 18N (high part)
  float* ecyclo = nullptr;   // its low part: the correction is kept in double-float
  float* f = nullptr;        // loads, 18N (high part)
  float* flo = nullptr;      // low part of the double-float loads, 18N
  float* r = nullptr;        // CG residual, 18N
  float* z = nullptr;        // preconditioned residual, 18N
  float* pv = nullptr;       // CG direction, 18N
  float* q = nullptr;        // K p and V-cycle level-0 residual scratch, 18N
  float* tmp = nullptr;      // N floats scratch (OC)

  int nlev = 0;
  homo::Level lev[homo::kMaxLevels];
  std::vector<float> hBf;    // level-1 Galerkin tables (host), 8 * 576 floats
  int nc = 0, mc = 0;        // coarsest cells per axis, 3*nc^3
  double* A = nullptr;       // mc*mc FP64 work (coarsest)
  double* G = nullptr;       // mc*mc FP64 centred pseudo-inverse of the coarsest operator

  double* part = nullptr;    // reduction partials
  size_t part_cap = 0;       // doubles
  double* scal = nullptr;    // device slots (homo::Slot)
  double* hscal = nullptr;   // pinned host mirror of scal

  bool loads_valid = false, hier_valid = false, solved = false, density_set = false;
  std::string err;

  // measurement: launch counter and optional per-class event timing
  struct ProfRec {
    int kc;
    cudaEvent_t a, b;
  };
  long long launches = 0;
  bool prof = false;
  std::vector<ProfRec> pending;
  std::vector<cudaEvent_t> event_pool;
  long long prof_n[HOMO_KC_COUNT] = {};
  double prof_ms[HOMO_KC_COUNT] = {};

  // relative residual of the 6 cases after every CG iteration of the last solve
  std::vector<double> history;

  // Chebyshev smoother: upper end of the spectrum of D^-1 K per smoothed level
  double lam[homo::kMaxLevels] = {};

  // CUDA graphs of one CG iteration (index: first iteration of a cycle or not), captured
  // on first use after the hierarchy is built and dropped when it is rebuilt
  // fine Gauss-Seidel variant: load cases per thread (3 or 6) and threads per block
  // (128 or 256); set by homo_set_tuning / homo_autotune
  int gs_cases = 3, gs_block = 256;
  // coarse Gauss-Seidel kernels (homo_set_coarse_smoother): levels with at most gs_fuse_n
  // cells per axis run every sweep of a smoothing phase as one thread-block-cluster launch,
  // levels with at most gs_split_n one launch per colour with a thread per (vertex, case),
  // larger levels one launch per colour with a thread per vertex; gs_cluster: the largest
  // cluster the device launches (-1: none, per-colour launches everywhere)
  int gs_fuse_n = 32, gs_split_n = 32, gs_cluster = -1;
  // levels with at most gs_res_n cells per axis (FP32 stencils, shared memory permitting)
  // keep each case's displacement resident in the clusters' shared memory instead;
  // gs_resident: the largest cluster of that form the device launches (-1: none)
  int gs_res_n = 16, gs_resident = -1;

  cudaGraphExec_t cg_graph[2] = {nullptr, nullptr};
  long long cg_graph_launches[2] = {0, 0};   // kernels per replay
  double cg_graph_tol = 0.0;                  // inner tolerance captured in the graphs
};

namespace homo {

// ---- host helpers (element.cu) ----
void build_element_matrix(double nu, KeParam& ke, LoadParam& ld, ChiParam& chi);
void build_level1_tables(const KeParam& ke, float* host_Bf /* 8*576 */);
int build_filter_param(double radius, FilterParam& fp);

// ---- warm-start network convolution on the tcgen05 tensor cores (conv_tc.cu) ----
cudaError_t conv3d_tc(int n, int cin, int epi, const void* x, const void* w, const float* bias, const void* res,
                      const void* mask, void* out, float* outf, const double* scale, cudaStream_t s);
int conv3d_tc_take_timeouts();
cudaError_t conv3d_tc_wait_probe(int blocks);

// ---- launchers (fine.cu) ----
cudaError_t launch_simp(const float* rho_in, float* rho_out, float* E, size_t N, float p,
                        float E0, float Emin, cudaStream_t s);
cudaError_t launch_loads(const homo_ctx* c, float* f);
// out = K u on level 0 in difference form; if part != nullptr also block partials of the
// dots (u_c, out_c) and the 18 plane sums of out (24 doubles per block; *grid_out blocks).
cudaError_t launch_fine_apply(const homo_ctx* c, const float* u, float* out, double* part,
                              int* grid_out);
// tiled finest-level stencil (fine_tiled.cu): mode 1 = launch_fine_apply; 2 = b - K (u + ulo)
// in difference form from both parts, with norms (FP32 true residual); 3 = (b - bmean) - K u;
// 4 = u + c0 S^-1 (b - bmean - K u); 5 = u + c0 (u - out) + c1 S^-1 (b - bmean - K u), in
// place on out; 6 = (1 + c0) u + c1 S^-1 (b - bmean - K u) (Chebyshev steps)
cudaError_t launch_fine_tiled(const homo_ctx* c, int mode, const float* u, const float* b, float* out,
                              double* part, int* grid_out, const double* bmean = nullptr,
                              float c0 = 0.f, float c1 = 0.f, const float* ulo = nullptr);
// out = c0 S^-1 (b - bmean) pointwise on level 0 (first Chebyshev step from zero)
cudaError_t launch_fine_jacobi_start(const homo_ctx* c, const float* b, const double* bmean, float* out,
                                     float c0);
// coarse Chebyshev step with the stored stencil: x_in == null means x_in = 0;
// mode 0: out = x_in + c0 S^-1 (b - K x_in); mode 1: out = x_in + c0 (x_in - out) + c1 S^-1 (b - K x_in);
// mode 3: out = (1 + c0) x_in + c1 S^-1 (b - K x_in)
cudaError_t launch_coarse_cheb(const Level& L, const float* b, const float* x_in, float* out, int mode,
                               float c0, float c1, cudaStream_t s);
// y = S^-1 K x on a stored-stencil level (power iteration for the Chebyshev interval)
cudaError_t launch_coarse_dinvk(const Level& L, const float* x, float* y, cudaStream_t s);
// mixed precision: L.sth = symmetrised BF16 copy of L.st
cudaError_t launch_stencil_bf16(const Level& L, cudaStream_t s);
cudaError_t launch_fill_hash(float* x, size_t count, unsigned seed, cudaStream_t s);
// largest eigenvalue of blockdiag(K0)^-1 K0 (host arithmetic)
double element_jacobi_bound(const KeParam& ke);
// symmetric n x n eigen-decomposition (n <= 8), double: a -> diag, columns of v eigenvectors
void sym_eigen(int n, double* a, double* v);
size_t tiled_smem_bytes(int mode);
// dynamic shared-memory limit of every tiled mode on the current device (before any capture)
cudaError_t tiled_init();
int tiled_grid_blocks(int n);
// ulo != null: out = (b + flo) - K (u + ulo) in double-float (b must be the loads f; accurate true residual) with
// partials of ||out_c||^2 and plane sums; ulo == null: out = (b - bmean) - K u (bmean: 18
// plane means or null).
cudaError_t launch_fine_residual(const homo_ctx* c, const float* b, const float* u,
                                 const float* ulo, float* out, double* part, int* grid_out,
                                 const double* bmean);
// first != 0: first sweep from u = 0, colours 0..7 (u need not be cleared); fmean: plane
// means subtracted from f, or null
cudaError_t launch_fine_gs(const homo_ctx* c, int colour, const float* f, float* u, int first,
                           const double* fmean);
// (cases, block) is a compiled variant of the fine Gauss-Seidel kernel
bool gs_variant_ok(int cases, int block);
cudaError_t launch_fine_elem(const homo_ctx* c, int mode, const double* g36, float* sens,
                             double* part, int* grid_out);

// ---- launchers (coarse.cu) ----
cudaError_t launch_level1_assemble(const homo_ctx* c, const Level& L1);
// Galerkin product of level Lf into Lc, one axis at a time; tmp1 (>= 243 n^3 / 2 floats)
// and tmp2 (>= 243 n^3 / 4) hold the two intermediate stencils (n = Lf.n).
cudaError_t launch_galerkin(const Level& Lf, const Level& Lc, float* tmp1, float* tmp2, cudaStream_t s);
cudaError_t launch_coarse_residual(const Level& L, const float* b, const float* x, float* out,
                                   cudaStream_t s);
cudaError_t launch_coarse_gs(const Level& L, int colour, const float* f, float* x, int first,
                             cudaStream_t s);
// Every sweep of one smoothing phase of level L (sweeps 8-colour sweeps, colours 7..0 when
// reverse, the first from x = 0 when first) as one launch of a thread-block cluster of at
// most cluster_max CTAs; bitwise the iterates of the per-colour launches.
cudaError_t launch_coarse_gs_sweeps(const Level& L, int sweeps, int reverse, int first, const float* f,
                                    float* x, int cluster_max, cudaStream_t s);
// One colour pass of level L with a thread per (vertex, case); bitwise launch_coarse_gs.
cudaError_t launch_coarse_gs_item(const Level& L, int colour, const float* f, float* x, int first,
                                  cudaStream_t s);
// Every sweep of one smoothing phase of level L with each case's displacement resident in
// shared memory (FP32 stencils only; coarse_resident_ok says whether L qualifies with
// clusters of at most cluster_max CTAs); bitwise the iterates of the per-colour launches.
cudaError_t launch_coarse_gs_resident(const Level& L, int sweeps, int reverse, int first, const float* f,
                                      float* x, int cluster_max, cudaStream_t s);
bool coarse_resident_ok(const Level& L, int cluster_max);
// Largest cluster of the resident form the current device launches (-1: none).
int coarse_resident_size();
// Largest cluster (16, 8 or 4 CTAs) the fused smoother can launch on the current device,
// -1 when none; queried once per device.
int coarse_cluster_size();
cudaError_t launch_restrict(int nf, const float* fine, float* coarse, cudaStream_t s);
cudaError_t launch_prolong_add(int nf, const float* coarse, float* fine, int overwrite,
                               cudaStream_t s);
cudaError_t launch_coarsest_setup(homo_ctx* c);
cudaError_t launch_coarsest_apply(const homo_ctx* c, const float* b, float* x);
cudaError_t launch_stencil_export(const Level& L, float* out, cudaStream_t s);
// level-0 stencil (243 planes, colour-blocked when n is even) built from E and K0
cudaError_t launch_fine_stencil(const homo_ctx* c, const Level& L0);

// ---- launchers (learned.cu): warm-start network layers (layouts in homo.h) ----
// scale: 6 per-case factors of the planes epilogues (host, nullable = 1)
cudaError_t nn_conv3d(int n, int cin, const void* x, const void* w, const float* bias, const void* res,
                      const void* mask, int epi, void* out, float* outf, const double* scale, cudaStream_t s);
// scratch: homo_nn_wgrad_scratch(n, cin) floats
cudaError_t nn_wgrad(int n, int cin, const void* x, const void* dy, float* dw, float* db, float* scratch,
                     cudaStream_t s);
cudaError_t nn_features(int n, const float* rho, void* x, cudaStream_t s);
// part: HOMO_NN_MSE_SCRATCH - 1 doubles; *nblk partials written
cudaError_t nn_mse(int n, const float* y, const float* u, const double* scale, void* dy, double* part, int* nblk,
                   cudaStream_t s);
cudaError_t nn_adam(size_t count, float* w, const float* g, float* m, float* v, int step, double lr, double b1,
                    double b2, double eps, cudaStream_t s);
cudaError_t nn_pack(int cin, const float* w, void* wf, void* wb, cudaStream_t s);
cudaError_t nn_pool(int n, int f, const float* rho, float* out, cudaStream_t s);

// ---- launchers (vec.cu) ----
int reduce_grid(size_t n_items);
cudaError_t launch_sum_partials(const double* part, int nblk, int nv, double* out,
                                cudaStream_t s);
cudaError_t launch_dot6(const float* a, const float* b, size_t N, double* part, int* grid_out,
                        cudaStream_t s);
// (r - rmean, z) per case and plane sums of z; rmean: 18 doubles or null
cudaError_t launch_dot6_zsum(const float* r, const float* z, size_t N, const double* rmean,
                             double* part, int* grid_out, cudaStream_t s);
cudaError_t launch_cg_alpha(double* scal, cudaStream_t s);
cudaError_t launch_cg_beta(double* scal, int first, cudaStream_t s);
// centred norms and plane means of r from its raw sums, active flags
cudaError_t launch_cg_active(double* scal, double tol, size_t N, cudaStream_t s);
// e += alpha p, r -= alpha (q - mean q), partials of ||r||^2 and plane sums of r
cudaError_t launch_cg_update_er(float* e, float* elo, float* r, const float* p, const float* q,
                                const double* scal, size_t N, double* part, int* grid_out,
                                cudaStream_t s);
// (u, ulo) += e in double-float, e = 0
cudaError_t launch_fold(float* u, float* ulo, float* e, float* elo, size_t n, cudaStream_t s);
cudaError_t launch_cg_update_p(float* p, const float* z, const double* scal, size_t N,
                               cudaStream_t s);
cudaError_t launch_split_set(float* hi, float* lo, const float* src, size_t n, cudaStream_t s);
cudaError_t launch_split_get(const float* hi, const float* lo, float* dst, size_t n,
                             cudaStream_t s);
// Orbit averages of an n^3 element field under the group (in may equal out).
cudaError_t launch_symmetrize(const SymParam& sp, int n, const float* in, float* out, cudaStream_t s);
int build_sym_param(int kind, SymParam& sp);
// y_e = sum over Q_n of w_a Q_a(centre_e) (FP64) into y
cudaError_t launch_trig_basis(const TrigParam& tp, int n, double* y, cudaStream_t s);
// per-block sums of S(y - mu_c) for kTrigCand shifts mu_c = mu0 + c * dmu (nv = kTrigCand)
cudaError_t launch_trig_volume(const double* y, size_t N, double mu0, double dmu, double k, double Vh,
                               double rho_min, double* part, int* grid_out, cudaStream_t s);
cudaError_t launch_trig_project(const double* y, size_t N, double mu, double k, double Vh, double rho_min,
                                float* rho, cudaStream_t s);
cudaError_t launch_filter(const FilterParam& fp, int n, const float* in, float* out,
                          cudaStream_t s);
// density-weighted sensitivity filter (out must alias neither rho nor dc)
cudaError_t launch_sensitivity_filter(const FilterParam& fp, int n, const float* rho, const float* dc,
                                      float gamma, float* out, cudaStream_t s);
cudaError_t launch_oc(homo_ctx* c, const float* dc, float* rho, double volfrac, double move,
                      double eta, double rho_min, double* change);

}  // namespace homo
