// Host side of the batched solve (include/dd_tv.h, dd_tv_batch_*): one arena holding
// the state of every image, per-image descriptors on the device, and the two batched
// launches per outer iteration (interface multipliers, local solves), captured into
// CUDA graphs.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "../../include/dd_tv.h"
#include "internal.cuh"

using namespace ddtv;

namespace {
thread_local char g_batch_create_err[512] = {0};
constexpr int kMaxGraphs = 8;  // captured run lengths kept per batch (least recently used dropped)
}  // namespace

struct dd_tv_batch {
  int n = 0;
  dd_tv_batch_params p{};
  std::vector<dd_tv_batch_image> img;
  std::vector<LocalArgs> host_args;  // per image, pointers into the arena
  std::vector<Strips> host_strips;   // 2 per image
  std::vector<int> fid, tile_base, elem_base;
  std::vector<float> sigma;
  int total_tiles = 0, total4 = 0;
  long long pixels = 0;
  char* arena = nullptr;
  size_t arena_bytes = 0;
  LocalArgs* d_args = nullptr;
  Strips* d_strips = nullptr;
  int *d_fid = nullptr, *d_tile_img = nullptr, *d_tile_base = nullptr, *d_elem_base = nullptr;
  float* d_sigma = nullptr;
  int* d_err = nullptr;
  double* partials = nullptr;
  unsigned int* counter = nullptr;
  double* red_out = nullptr;
  cudaStream_t stream = nullptr, own = nullptr;
  int outer = 0;
  bool loaded = false;
  // one CUDA graph per (outer iterations, start parity) of dd_tv_batch_iterate calls:
  // a call of n > 1 outer iterations is one graph launch
  struct Run {
    int count, par;
    cudaGraphExec_t exec;
    long long used;
  };
  std::vector<Run> graphs;
  long long tick = 0;
  char err[512] = {0};
};

namespace {

int bfail(dd_tv_batch* b, int code, const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(b ? b->err : g_batch_create_err, 512, fmt, ap);
  va_end(ap);
  return code;
}

#define BCK(call)                                                                                     \
  do {                                                                                                \
    cudaError_t e_ = (call);                                                                          \
    if (e_ != cudaSuccess) return bfail(b, DD_TV_ECUDA, "%s: %s", #call, cudaGetErrorString(e_));    \
  } while (0)

size_t align_up(size_t x) { return (x + 255) & ~(size_t)255; }

void coefs_for(const dd_tv_batch_params& p, double alpha, double tau, double gamma, std::vector<Coef>& c) {
  const int K = p.inner_iters;
  c.resize(K);
  double tk = p.tau0, sk = p.sigma0;
  for (int k = 0; k < K; ++k) {
    const double th = 1.0 / std::sqrt(1.0 + 2.0 * gamma * tk);
    c[k] = Coef{(float)sk,
                (float)(1.0 / (1.0 + sk * alpha)),
                (float)(sk * alpha / (1.0 + sk * alpha)),
                (float)(sk * alpha),
                (float)(tau / (tau + tk)),
                (float)(tau * tk / (tau + tk)),
                (float)(tk / (tau + tk)),
                (float)th};
    tk = th * tk;
    sk = sk / th;
  }
}

cudaError_t outer_once(dd_tv_batch* b, int par) {
  BatchIfaceArgs ia;
  ia.args = b->d_args;
  ia.strips = b->d_strips;
  ia.sigma = b->d_sigma;
  ia.elem_base = b->d_elem_base;
  ia.n_img = b->n;
  ia.cur_set = par;
  cudaError_t e = launch_interface_batch(ia, b->total4, b->stream);
  if (e != cudaSuccess) return e;
  BatchArgs ba;
  ba.args = b->d_args;
  ba.strips = b->d_strips;
  ba.fid = b->d_fid;
  ba.tile_img = b->d_tile_img;
  ba.tile_base = b->d_tile_base;
  ba.write_set = 1 - par;
  return launch_fused_batch(ba, b->total_tiles, b->p.tile, b->p.variant, b->p.inner_iters, b->stream);
}

void drop_batch_graphs(dd_tv_batch* b) {
  for (auto& r : b->graphs) cudaGraphExecDestroy(r.exec);
  b->graphs.clear();
}

int run(dd_tv_batch* b, int count) {
  if (count <= 0) return DD_TV_OK;
  const int par = b->outer & 1;
  if (count == 1) {
    BCK(outer_once(b, par));
    b->outer += 1;
    return DD_TV_OK;
  }
  cudaGraphExec_t exec = nullptr;
  for (auto& r : b->graphs)
    if (r.count == count && r.par == par) {
      exec = r.exec;
      r.used = ++b->tick;
    }
  if (!exec) {
    cudaGraph_t graph = nullptr;
    BCK(cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
    cudaError_t e = cudaSuccess;
    for (int q = 0; q < count && e == cudaSuccess; ++q) e = outer_once(b, (par + q) & 1);
    cudaError_t e2 = cudaStreamEndCapture(b->stream, &graph);
    if (e != cudaSuccess || e2 != cudaSuccess) {
      if (graph) cudaGraphDestroy(graph);
      return bfail(b, DD_TV_ECUDA, "graph capture: %s", cudaGetErrorString(e != cudaSuccess ? e : e2));
    }
    e = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return bfail(b, DD_TV_ECUDA, "cudaGraphInstantiate: %s", cudaGetErrorString(e));
    if ((int)b->graphs.size() >= kMaxGraphs) {  // drop the least recently used run length
      size_t lru = 0;
      for (size_t q = 1; q < b->graphs.size(); ++q)
        if (b->graphs[q].used < b->graphs[lru].used) lru = q;
      cudaGraphExecDestroy(b->graphs[lru].exec);
      b->graphs.erase(b->graphs.begin() + lru);
    }
    b->graphs.push_back(dd_tv_batch::Run{count, par, exec, ++b->tick});
  }
  BCK(cudaGraphLaunch(exec, b->stream));
  b->outer += count;
  return DD_TV_OK;
}

}  // namespace

extern "C" {

int dd_tv_batch_create(dd_tv_batch** out, const dd_tv_batch_image* images, int n, const dd_tv_batch_params* p) {
  if (!out) return DD_TV_EINVAL;
  *out = nullptr;
  dd_tv_batch* b = nullptr;
  if (!images || n < 1 || !p) return bfail(nullptr, DD_TV_EINVAL, "need n >= 1 images and params");
  if (p->tile != 128 && p->tile != 64)
    return bfail(nullptr, DD_TV_EUNSUPPORTED, "batched subdomain side must be 64 or 128 (got %d)", p->tile);
  const int T = p->tile;
  if (p->inner_iters < 1 || p->inner_iters > DD_TV_MAX_INNER) return bfail(nullptr, DD_TV_EINVAL, "bad inner_iters");
  if (!(p->tau0 > 0) || !(p->sigma0 > 0) || p->tau0 * p->sigma0 > 0.125 * (1 + 1e-12))
    return bfail(nullptr, DD_TV_EINVAL, "tau0, sigma0 must be > 0 with tau0 sigma0 <= 1/8");
  if (p->variant != 0 && !(p->variant == 2 && p->tile == 128))
    return bfail(nullptr, DD_TV_EINVAL, "batch variant must be 0 (or 2 with 128 x 128 subdomains)");
  for (int i = 0; i < n; ++i) {
    const dd_tv_batch_image& m = images[i];
    if (m.height < T || m.width < T || m.height % T || m.width % T)
      return bfail(nullptr, DD_TV_EINVAL, "image %d: sides must be positive multiples of the subdomain side %d (got "
                   "%d x %d)", i, T, m.height, m.width);
    if (m.fidelity < DD_TV_L2 || m.fidelity > DD_TV_SEG) return bfail(nullptr, DD_TV_EINVAL, "image %d: fidelity", i);
    if (!(m.alpha > 0) || !std::isfinite(m.alpha)) return bfail(nullptr, DD_TV_EINVAL, "image %d: alpha", i);
    if (m.tau > 0 && (!(m.sigma > 0) || m.tau * m.sigma > 0.5 * (1 + 1e-12)))
      return bfail(nullptr, DD_TV_EINVAL, "image %d: need sigma > 0 and tau sigma <= 1/2", i);
    if ((long long)m.height * m.width > (1LL << 31) - 1) return bfail(nullptr, DD_TV_EINVAL, "image %d too large", i);
  }
  b = new (std::nothrow) dd_tv_batch();
  if (!b) return DD_TV_ENOMEM;
  b->n = n;
  b->p = *p;
  b->img.assign(images, images + n);
  cudaError_t e = fused_prepare();
  if (e != cudaSuccess) {
    bfail(nullptr, DD_TV_ECUDA, "fused kernel set-up: %s", cudaGetErrorString(e));
    delete b;
    return DD_TV_ECUDA;
  }
  // arena layout: per image f, u, P1, P2, lamh, lamv, 2 strip sets, coefficients
  std::vector<size_t> off_f(n), off_u(n), off_p1(n), off_p2(n), off_lh(n), off_lv(n), off_st(n), off_co(n);
  std::vector<std::vector<Coef>> coefs(n);
  size_t at = 0;
  for (int i = 0; i < n; ++i) {
    const dd_tv_batch_image& m = b->img[i];
    const int NR = m.height / T, NC = m.width / T;
    const size_t npx = (size_t)m.height * m.width, n1 = (size_t)(m.height + NR) * m.width,
                 n2 = (size_t)m.height * (m.width + NC), nh = (size_t)(NR - 1) * m.width, nv = (size_t)(NC - 1) * m.height;
    off_f[i] = at; at = align_up(at + 4 * npx);
    off_u[i] = at; at = align_up(at + 4 * npx);
    off_p1[i] = at; at = align_up(at + 4 * n1);
    off_p2[i] = at; at = align_up(at + 4 * n2);
    off_lh[i] = at; at = align_up(at + 4 * nh);
    off_lv[i] = at; at = align_up(at + 4 * nv);
    off_st[i] = at; at = align_up(at + 4 * 4 * (nh + nv));
    const double tau = m.tau > 0 ? m.tau : (m.fidelity == DD_TV_SEG ? 1.0 : 50.0);
    coefs_for(b->p, m.alpha, tau, 1.0 / (8.0 * tau), coefs[i]);
    off_co[i] = at; at = align_up(at + sizeof(Coef) * coefs[i].size());
  }
  b->arena_bytes = at;
  if ((e = cudaMalloc((void**)&b->arena, at)) != cudaSuccess) {
    bfail(nullptr, DD_TV_ENOMEM, "cudaMalloc(%zu bytes) for the batch state: %s", at, cudaGetErrorString(e));
    delete b;
    return DD_TV_ENOMEM;
  }
  b->host_args.resize(n);
  b->host_strips.resize(2 * n);
  b->fid.resize(n);
  b->sigma.resize(n);
  b->tile_base.resize(n);
  b->elem_base.resize(n + 1);
  std::vector<int> tile_img;
  int tb = 0, eb = 0;
  for (int i = 0; i < n; ++i) {
    const dd_tv_batch_image& m = b->img[i];
    const int NR = m.height / T, NC = m.width / T;
    const size_t nh = (size_t)(NR - 1) * m.width, nv = (size_t)(NC - 1) * m.height;
    const double tau = m.tau > 0 ? m.tau : (m.fidelity == DD_TV_SEG ? 1.0 : 50.0);
    const double sigma = m.tau > 0 ? m.sigma : 0.5 / tau;
    LocalArgs& A = b->host_args[i];
    A.g = Grid{m.height, m.width, NR, NC};
    A.K = p->inner_iters;
    A.tau = (float)tau;
    A.c1 = (float)m.c1;
    A.c2 = (float)m.c2;
    A.f = (const float*)(b->arena + off_f[i]);
    A.mask = nullptr;
    A.u = (float*)(b->arena + off_u[i]);
    A.P1 = (float*)(b->arena + off_p1[i]);
    A.P2 = (float*)(b->arena + off_p2[i]);
    A.lamh = (const float*)(b->arena + off_lh[i]);
    A.lamv = (const float*)(b->arena + off_lv[i]);
    A.coef = (const Coef*)(b->arena + off_co[i]);
    A.out = Strips{};
    for (int s = 0; s < 2; ++s) {
      float* base = (float*)(b->arena + off_st[i]) + (size_t)s * 2 * (nh + nv);
      b->host_strips[2 * i + s] = Strips{base, base + nh, base + 2 * nh, base + 2 * nh + nv};
    }
    b->fid[i] = m.fidelity;
    b->sigma[i] = (float)sigma;
    b->tile_base[i] = tb;
    for (int t = 0; t < NR * NC; ++t) tile_img.push_back(i);
    tb += NR * NC;
    b->elem_base[i] = eb;
    eb += (int)((nh + nv) / 4);
    b->pixels += (long long)m.height * m.width;
  }
  b->elem_base[n] = eb;
  b->total_tiles = tb;
  b->total4 = eb;
  b->stream = nullptr;
  if ((e = cudaMalloc((void**)&b->d_args, sizeof(LocalArgs) * n)) != cudaSuccess ||
      (e = cudaMalloc((void**)&b->d_strips, sizeof(Strips) * 2 * n)) != cudaSuccess ||
      (e = cudaMalloc((void**)&b->d_fid, sizeof(int) * n)) != cudaSuccess ||
      (e = cudaMalloc((void**)&b->d_tile_img, sizeof(int) * tb)) != cudaSuccess ||
      (e = cudaMalloc((void**)&b->d_tile_base, sizeof(int) * n)) != cudaSuccess ||
      (e = cudaMalloc((void**)&b->d_elem_base, sizeof(int) * (n + 1))) != cudaSuccess ||
      (e = cudaMalloc((void**)&b->d_sigma, sizeof(float) * n)) != cudaSuccess ||
      (e = cudaMalloc((void**)&b->d_err, sizeof(int))) != cudaSuccess ||
      (e = cudaMalloc((void**)&b->partials, sizeof(double) * reduce_partials_count())) != cudaSuccess ||
      (e = cudaMalloc((void**)&b->counter, sizeof(unsigned int))) != cudaSuccess ||
      (e = cudaMalloc((void**)&b->red_out, 2 * sizeof(double))) != cudaSuccess) {
    bfail(nullptr, DD_TV_ENOMEM, "batch descriptors: %s", cudaGetErrorString(e));
    dd_tv_batch_destroy(b);
    return DD_TV_ENOMEM;
  }
  for (int i = 0; i < n; ++i) b->host_args[i].err = b->d_err;
  if ((e = cudaMemcpy(b->d_args, b->host_args.data(), sizeof(LocalArgs) * n, cudaMemcpyHostToDevice)) ||
      (e = cudaMemcpy(b->d_strips, b->host_strips.data(), sizeof(Strips) * 2 * n, cudaMemcpyHostToDevice)) ||
      (e = cudaMemcpy(b->d_fid, b->fid.data(), sizeof(int) * n, cudaMemcpyHostToDevice)) ||
      (e = cudaMemcpy(b->d_tile_img, tile_img.data(), sizeof(int) * tb, cudaMemcpyHostToDevice)) ||
      (e = cudaMemcpy(b->d_tile_base, b->tile_base.data(), sizeof(int) * n, cudaMemcpyHostToDevice)) ||
      (e = cudaMemcpy(b->d_elem_base, b->elem_base.data(), sizeof(int) * (n + 1), cudaMemcpyHostToDevice)) ||
      (e = cudaMemcpy(b->d_sigma, b->sigma.data(), sizeof(float) * n, cudaMemcpyHostToDevice)) ||
      (e = cudaMemset(b->d_err, 0, sizeof(int))) || (e = cudaMemset(b->counter, 0, sizeof(unsigned int))) ||
      (e = cudaStreamCreate(&b->own))) {
    bfail(nullptr, DD_TV_ECUDA, "batch set-up: %s", cudaGetErrorString(e));
    dd_tv_batch_destroy(b);
    return DD_TV_ECUDA;
  }
  for (int i = 0; i < n; ++i) {
    if ((e = cudaMemcpy((void*)b->host_args[i].coef, coefs[i].data(), sizeof(Coef) * coefs[i].size(),
                        cudaMemcpyHostToDevice)) != cudaSuccess) {
      bfail(nullptr, DD_TV_ECUDA, "batch coefficients: %s", cudaGetErrorString(e));
      dd_tv_batch_destroy(b);
      return DD_TV_ECUDA;
    }
  }
  b->stream = b->own;
  *out = b;
  return DD_TV_OK;
}

int dd_tv_batch_destroy(dd_tv_batch* b) {
  if (!b) return DD_TV_OK;
  drop_batch_graphs(b);
  void* bufs[] = {b->arena, b->d_args, b->d_strips, b->d_fid, b->d_tile_img, b->d_tile_base, b->d_elem_base,
                  b->d_sigma, b->d_err, b->partials, b->counter, b->red_out};
  for (void* q : bufs)
    if (q) cudaFree(q);
  if (b->own) cudaStreamDestroy(b->own);
  delete b;
  return DD_TV_OK;
}

const char* dd_tv_batch_last_error(const dd_tv_batch* b) { return b ? b->err : g_batch_create_err; }

int dd_tv_batch_set_stream(dd_tv_batch* b, void* stream) {
  if (!b) return DD_TV_EINVAL;
  b->stream = stream ? (cudaStream_t)stream : b->own;
  return DD_TV_OK;
}

int dd_tv_batch_load(dd_tv_batch* b, const float* const* f_dev) {
  if (!b) return DD_TV_EINVAL;
  if (!f_dev) return bfail(b, DD_TV_EINVAL, "f_dev is NULL");
  for (int i = 0; i < b->n; ++i) {
    if (!f_dev[i]) return bfail(b, DD_TV_EINVAL, "f_dev[%d] is NULL", i);
    const LocalArgs& A = b->host_args[i];
    const size_t npx = (size_t)A.g.H * A.g.W, n1 = (size_t)(A.g.H + A.g.NR) * A.g.W,
                 n2 = (size_t)A.g.H * (A.g.W + A.g.NC), nh = (size_t)(A.g.NR - 1) * A.g.W,
                 nv = (size_t)(A.g.NC - 1) * A.g.H;
    BCK(cudaMemcpyAsync((void*)A.f, f_dev[i], 4 * npx, cudaMemcpyDeviceToDevice, b->stream));
    BCK(launch_init_u(A.g, b->fid[i], A.f, nullptr, A.u, b->stream));
    BCK(cudaMemsetAsync(A.P1, 0, 4 * n1, b->stream));
    BCK(cudaMemsetAsync(A.P2, 0, 4 * n2, b->stream));
    if (nh) BCK(cudaMemsetAsync((void*)A.lamh, 0, 4 * nh, b->stream));
    if (nv) BCK(cudaMemsetAsync((void*)A.lamv, 0, 4 * nv, b->stream));
    if (nh + nv) BCK(cudaMemsetAsync(b->host_strips[2 * i].SB, 0, 4 * 4 * (nh + nv), b->stream));
  }
  b->outer = 0;
  b->loaded = true;
  return DD_TV_OK;
}

int dd_tv_batch_iterate(dd_tv_batch* b, int n_outer) {
  if (!b) return DD_TV_EINVAL;
  if (!b->loaded) return bfail(b, DD_TV_EINVAL, "no data loaded");
  if (n_outer < 0) return bfail(b, DD_TV_EINVAL, "n_outer must be >= 0");
  return run(b, n_outer);
}

int dd_tv_batch_get_u(dd_tv_batch* b, int i, float* u_dev) {
  if (!b) return DD_TV_EINVAL;
  if (i < 0 || i >= b->n || !u_dev) return bfail(b, DD_TV_EINVAL, "bad image index or pointer");
  const LocalArgs& A = b->host_args[i];
  BCK(cudaMemcpyAsync(u_dev, A.u, 4 * (size_t)A.g.H * A.g.W, cudaMemcpyDeviceToDevice, b->stream));
  return DD_TV_OK;
}

int dd_tv_batch_energy(dd_tv_batch* b, int i, double* J_out) {
  if (!b) return DD_TV_EINVAL;
  if (i < 0 || i >= b->n || !J_out) return bfail(b, DD_TV_EINVAL, "bad image index or pointer");
  const LocalArgs& A = b->host_args[i];
  BCK(launch_energy(A.g, b->fid[i], (float)b->img[i].alpha, A.c1, A.c2, A.u, A.f, nullptr, nullptr, nullptr,
                    b->partials, b->counter, b->red_out, b->stream));
  double o[2];
  BCK(cudaMemcpyAsync(o, b->red_out, sizeof(o), cudaMemcpyDeviceToHost, b->stream));
  BCK(cudaStreamSynchronize(b->stream));
  int flag = 0;
  BCK(cudaMemcpy(&flag, b->d_err, sizeof(int), cudaMemcpyDeviceToHost));
  if (flag) return bfail(b, DD_TV_ETIMEOUT, "a device-side wait ran out (results are invalid)");
  *J_out = o[0];
  return DD_TV_OK;
}

long long dd_tv_batch_pixels(const dd_tv_batch* b) { return b ? b->pixels : -1; }

}  // extern "C"
