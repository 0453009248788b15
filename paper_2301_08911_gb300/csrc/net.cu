// homo_net: the warm-start network as one native object (layer sequencing, parameter
// and Adam state, packed weights, activation arenas). Layer arithmetic is in learned.cu;
// the network and its layouts are described in homo.h.
#include <algorithm>
#include <string>
#include <vector>

#include "homo_internal.cuh"

using namespace homo;

namespace {

constexpr int kC = HOMO_NN_CHANNELS;
constexpr int kMaxBlocks = 16;
constexpr size_t kAlign = 256;

size_t round_up(size_t b) { return (b + kAlign - 1) / kAlign * kAlign; }

// One device allocation carved into aligned pieces.
struct Arena {
  char* base = nullptr;
  size_t size = 0;
  int n = 0;
  void release() {
    if (base) cudaFree(base);
    base = nullptr;
    size = 0;
    n = 0;
  }
};

}  // namespace

struct homo_net {
  int blocks = 0, layers = 0;
  size_t count = 0;
  std::vector<int> cin;
  std::vector<size_t> woff, boff, wbf_off, wbb_off;   // offsets (floats / bf16 elements)
  float* params = nullptr;
  float* grads = nullptr;
  float* m = nullptr;
  float* v = nullptr;
  __nv_bfloat16* wbf = nullptr;   // packed forward weights of every layer
  __nv_bfloat16* wbb = nullptr;   // packed transposed weights (layers with c_in = 32)
  int step = 0;
  cudaStream_t stream = nullptr;
  long long launches = 0;
  Arena pred, train;
  std::string err;

  const float* W(int l) const { return params + woff[l]; }
  const float* b(int l) const { return params + boff[l]; }
  const void* wf(int l) const { return wbf + wbf_off[l]; }
  const void* wb(int l) const { return wbb + wbb_off[l]; }
};

namespace {

int fail(homo_net* net, int st, const std::string& what) {
  net->err = what;
  return st;
}

int cuda_fail(homo_net* net, cudaError_t e, const char* where) {
  net->err = std::string(where) + ": " + cudaGetErrorString(e);
  return HOMO_ECUDA;
}

#define NN(net, call)                                         \
  do {                                                        \
    const cudaError_t e_ = (call);                            \
    if (e_ != cudaSuccess) return cuda_fail(net, e_, #call);  \
    ++(net)->launches;                                        \
  } while (0)

void layout(homo_net* net, int blocks) {
  net->blocks = blocks;
  net->layers = 2 * blocks + 2;
  net->cin.assign(net->layers, kC);
  net->cin[0] = HOMO_NN_FEATURES;
  size_t off = 0, fo = 0, bo = 0;
  for (int l = 0; l < net->layers; ++l) {
    const size_t nw = static_cast<size_t>(27) * kC * net->cin[l];
    net->woff.push_back(off);
    net->boff.push_back(off + nw);
    off += nw + kC;
    net->wbf_off.push_back(fo);
    fo += round_up(nw * 2) / 2;
    net->wbb_off.push_back(bo);
    if (net->cin[l] == kC) bo += round_up(nw * 2) / 2;
  }
  net->count = off;
}

size_t wbf_elems(const homo_net* net) {
  const int l = net->layers - 1;
  return net->wbf_off[l] + round_up(static_cast<size_t>(27) * kC * net->cin[l] * 2) / 2;
}

size_t wbb_elems(const homo_net* net) {
  const int l = net->layers - 1;
  return net->wbb_off[l] + round_up(static_cast<size_t>(27) * kC * kC * 2) / 2;
}

int pack_all(homo_net* net) {
  for (int l = 0; l < net->layers; ++l)
    NN(net, nn_pack(net->cin[l], net->W(l), net->wbf + net->wbf_off[l],
                    net->cin[l] == kC ? static_cast<void*>(net->wbb + net->wbb_off[l]) : nullptr, net->stream));
  return HOMO_OK;
}

int ensure_arena(homo_net* net, Arena& a, int n, size_t bytes) {
  if (a.base && a.n == n && a.size >= bytes) return HOMO_OK;
  a.release();
  if (cudaMalloc(reinterpret_cast<void**>(&a.base), bytes) != cudaSuccess) {
    cudaGetLastError();
    a.base = nullptr;
    return fail(net, HOMO_ENOMEM, "activation buffers: cudaMalloc failed");
  }
  a.size = bytes;
  a.n = n;
  return HOMO_OK;
}

struct Carve {
  char* p;
  template <class T>
  T* take(size_t bytes) {
    T* r = reinterpret_cast<T*>(p);
    p += round_up(bytes);
    return r;
  }
};

bool size_ok(int n) { return n >= 1 && n <= 1024; }

}  // namespace

extern "C" {

size_t homo_net_param_count(int blocks) {
  if (blocks < 1 || blocks > kMaxBlocks) return 0;
  homo_net tmp;
  layout(&tmp, blocks);
  return tmp.count;
}

int homo_net_create(homo_net** out, int blocks, const float* params) {
  if (!out || !params || blocks < 1 || blocks > kMaxBlocks) return HOMO_EINVAL;
  *out = nullptr;
  homo_net* net = new homo_net();
  layout(net, blocks);
  const size_t fb = net->count * sizeof(float);
  bool ok = cudaMalloc(reinterpret_cast<void**>(&net->params), fb) == cudaSuccess &&
            cudaMalloc(reinterpret_cast<void**>(&net->grads), fb) == cudaSuccess &&
            cudaMalloc(reinterpret_cast<void**>(&net->m), fb) == cudaSuccess &&
            cudaMalloc(reinterpret_cast<void**>(&net->v), fb) == cudaSuccess &&
            cudaMalloc(reinterpret_cast<void**>(&net->wbf), wbf_elems(net) * 2) == cudaSuccess &&
            cudaMalloc(reinterpret_cast<void**>(&net->wbb), wbb_elems(net) * 2) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    homo_net_destroy(net);
    return HOMO_ENOMEM;
  }
  ok = cudaMemcpy(net->params, params, fb, cudaMemcpyHostToDevice) == cudaSuccess &&
       cudaMemset(net->grads, 0, fb) == cudaSuccess && cudaMemset(net->m, 0, fb) == cudaSuccess &&
       cudaMemset(net->v, 0, fb) == cudaSuccess;
  if (!ok || pack_all(net) != HOMO_OK || cudaStreamSynchronize(net->stream) != cudaSuccess) {
    homo_net_destroy(net);
    return HOMO_ECUDA;
  }
  *out = net;
  return HOMO_OK;
}

int homo_net_destroy(homo_net* net) {
  if (!net) return HOMO_EINVAL;
  if (net->stream) cudaStreamSynchronize(net->stream);
  else cudaDeviceSynchronize();
  net->pred.release();
  net->train.release();
  for (void* p : {static_cast<void*>(net->params), static_cast<void*>(net->grads), static_cast<void*>(net->m),
                  static_cast<void*>(net->v), static_cast<void*>(net->wbf), static_cast<void*>(net->wbb)})
    if (p) cudaFree(p);
  delete net;
  return HOMO_OK;
}

const char* homo_net_last_error(const homo_net* net) { return net ? net->err.c_str() : "null network"; }

int homo_net_set_stream(homo_net* net, void* cuda_stream) {
  if (!net) return HOMO_EINVAL;
  net->stream = static_cast<cudaStream_t>(cuda_stream);
  return HOMO_OK;
}

int homo_net_get_params(homo_net* net, float* params) {
  if (!net || !params) return HOMO_EINVAL;
  const cudaError_t e = cudaMemcpyAsync(params, net->params, net->count * sizeof(float), cudaMemcpyDeviceToHost,
                                        net->stream);
  if (e != cudaSuccess) return cuda_fail(net, e, "homo_net_get_params");
  const cudaError_t f = cudaStreamSynchronize(net->stream);
  return f == cudaSuccess ? HOMO_OK : cuda_fail(net, f, "homo_net_get_params");
}

int homo_net_get_grads(homo_net* net, float* grads) {
  if (!net || !grads) return HOMO_EINVAL;
  const cudaError_t e = cudaMemcpyAsync(grads, net->grads, net->count * sizeof(float), cudaMemcpyDeviceToHost,
                                        net->stream);
  if (e != cudaSuccess) return cuda_fail(net, e, "homo_net_get_grads");
  const cudaError_t f = cudaStreamSynchronize(net->stream);
  return f == cudaSuccess ? HOMO_OK : cuda_fail(net, f, "homo_net_get_grads");
}

int homo_net_predict(homo_net* net, int n, const float* rho, const double* scale, float* u, int accumulate) {
  if (!net) return HOMO_EINVAL;
  if (!size_ok(n) || !rho || !u || !scale) return fail(net, HOMO_EINVAL, "homo_net_predict: bad argument");
  const size_t N = static_cast<size_t>(n) * n * n;
  const size_t bx = N * HOMO_NN_FEATURES * 2, ba = N * kC * 2;
  int st = ensure_arena(net, net->pred, n, round_up(bx) + 3 * round_up(ba));
  if (st != HOMO_OK) return st;
  Carve c{net->pred.base};
  void* X = c.take<char>(bx);
  void* A = c.take<char>(ba);
  void* B = c.take<char>(ba);
  void* T = c.take<char>(ba);
  cudaStream_t s = net->stream;
  NN(net, nn_features(n, rho, X, s));
  NN(net, nn_conv3d(n, HOMO_NN_FEATURES, X, net->wf(0), net->b(0), nullptr, nullptr, HOMO_NN_RELU, A, nullptr,
                    nullptr, s));
  for (int k = 0; k < net->blocks; ++k) {
    NN(net, nn_conv3d(n, kC, A, net->wf(1 + 2 * k), net->b(1 + 2 * k), nullptr, nullptr, HOMO_NN_RELU, T,
                      nullptr, nullptr, s));
    NN(net, nn_conv3d(n, kC, T, net->wf(2 + 2 * k), net->b(2 + 2 * k), A, nullptr, HOMO_NN_RELU, B, nullptr, nullptr,
                      s));
    std::swap(A, B);
  }
  const int lo = net->layers - 1;
  NN(net, nn_conv3d(n, kC, A, net->wf(lo), net->b(lo), nullptr, nullptr,
                    accumulate ? HOMO_NN_PLANES_ADD : HOMO_NN_PLANES, nullptr, u, scale, s));
  return HOMO_OK;
}

int homo_net_train_step(homo_net* net, int n, const float* rho, const float* u, const double* scale, double lr,
                        double* loss) {
  if (!net) return HOMO_EINVAL;
  bool sc_ok = scale != nullptr;
  for (int k = 0; sc_ok && k < 6; ++k) sc_ok = scale[k] > 0.0;
  if (!size_ok(n) || !rho || !u || !sc_ok || !(lr >= 0.0))
    return fail(net, HOMO_EINVAL, "homo_net_train_step: bad argument");
  const int B = net->blocks, lo = net->layers - 1;
  const size_t N = static_cast<size_t>(n) * n * n;
  const size_t bx = N * HOMO_NN_FEATURES * 2, ba = N * kC * 2, by = N * 18 * sizeof(float);
  const size_t scratch = homo_nn_wgrad_scratch(n, kC) * sizeof(float);
  const size_t bytes = round_up(bx) + (2 * B + 1 + 4) * round_up(ba) + round_up(by) + round_up(scratch) +
                       round_up(HOMO_NN_MSE_SCRATCH * sizeof(double));
  int st = ensure_arena(net, net->train, n, bytes);
  if (st != HOMO_OK) return st;
  Carve c{net->train.base};
  void* X = c.take<char>(bx);
  std::vector<void*> H(B + 1), T(B);
  for (auto& h : H) h = c.take<char>(ba);
  for (auto& t : T) t = c.take<char>(ba);
  void* G = c.take<char>(ba);
  void* S = c.take<char>(ba);
  void* S2 = c.take<char>(ba);
  void* Q = c.take<char>(ba);
  float* Y = c.take<float>(by);
  float* scr = c.take<float>(scratch);
  double* lbuf = c.take<double>(HOMO_NN_MSE_SCRATCH * sizeof(double));
  cudaStream_t s = net->stream;
  float* gr = net->grads;

  // forward, keeping every activation
  NN(net, nn_features(n, rho, X, s));
  NN(net, nn_conv3d(n, HOMO_NN_FEATURES, X, net->wf(0), net->b(0), nullptr, nullptr, HOMO_NN_RELU, H[0], nullptr,
                    nullptr, s));
  for (int k = 0; k < B; ++k) {
    NN(net, nn_conv3d(n, kC, H[k], net->wf(1 + 2 * k), net->b(1 + 2 * k), nullptr, nullptr, HOMO_NN_RELU, T[k],
                      nullptr, nullptr, s));
    NN(net, nn_conv3d(n, kC, T[k], net->wf(2 + 2 * k), net->b(2 + 2 * k), H[k], nullptr, HOMO_NN_RELU, H[k + 1],
                      nullptr, nullptr, s));
  }
  NN(net, nn_conv3d(n, kC, H[B], net->wf(lo), net->b(lo), nullptr, nullptr, HOMO_NN_PLANES, nullptr, Y, nullptr, s));

  // loss and its gradient
  int nblk = 0;
  NN(net, nn_mse(n, Y, u, scale, G, lbuf + 1, &nblk, s));
  NN(net, launch_sum_partials(lbuf + 1, nblk, 1, lbuf, s));

  // backward: s = dL/d(pre-activation of h_b), q = dL/d(pre-activation of t_b)
  NN(net, nn_wgrad(n, kC, H[B], G, gr + net->woff[lo], gr + net->boff[lo], scr, s));
  NN(net, nn_conv3d(n, kC, G, net->wb(lo), nullptr, nullptr, H[B], HOMO_NN_MASK, S, nullptr, nullptr, s));
  for (int k = B - 1; k >= 0; --k) {
    const int l1 = 1 + 2 * k, l2 = 2 + 2 * k;
    NN(net, nn_wgrad(n, kC, T[k], S, gr + net->woff[l2], gr + net->boff[l2], scr, s));
    NN(net, nn_conv3d(n, kC, S, net->wb(l2), nullptr, nullptr, T[k], HOMO_NN_MASK, Q, nullptr, nullptr, s));
    NN(net, nn_wgrad(n, kC, H[k], Q, gr + net->woff[l1], gr + net->boff[l1], scr, s));
    NN(net, nn_conv3d(n, kC, Q, net->wb(l1), nullptr, S, H[k], HOMO_NN_MASK, S2, nullptr, nullptr, s));
    std::swap(S, S2);
  }
  NN(net, nn_wgrad(n, HOMO_NN_FEATURES, X, S, gr + net->woff[0], gr + net->boff[0], scr, s));

  // update and repack
  net->step += 1;
  NN(net, nn_adam(net->count, net->params, gr, net->m, net->v, net->step, lr, 0.9, 0.999, 1e-8, s));
  st = pack_all(net);
  if (st != HOMO_OK) return st;
  if (loss) {
    cudaError_t e = cudaMemcpyAsync(loss, lbuf, sizeof(double), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(net, e, "homo_net_train_step: loss");
  }
  return HOMO_OK;
}

int homo_net_release(homo_net* net) {
  if (!net) return HOMO_EINVAL;
  if (net->stream) cudaStreamSynchronize(net->stream);
  else cudaDeviceSynchronize();
  net->pred.release();
  net->train.release();
  return HOMO_OK;
}

long long homo_net_launch_count(const homo_net* net) { return net ? net->launches : -1; }

}  // extern "C"
