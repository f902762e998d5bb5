// Host side of the dd_tv C ABI (include/dd_tv.h): argument validation, device
// state, the outer loop of Algorithm 1 on the three paths, CUDA-graph replay of the
// outer loop, state exchange and the energy/gap calls.
#include <algorithm>
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

constexpr int kGraphChunk = 4;  // outer iterations per captured graph (even: parity is preserved)

// message of the last failed dd_tv_create on this thread (no handle exists then)
thread_local char g_create_err[512] = {0};

}  // namespace

// Device memory of the reverse pass (dd_tv_adjoint_*).
struct AdjointWork {
  int N = 0, m = 0, nck = 0;     // outer iterations, checkpoint spacing, checkpoints
  long long gen = -1;            // load generation the checkpoints belong to
  size_t slot = 0;               // floats per saved state
  int cap_ck = 0, cap_seg = 0;   // saved-state slots allocated
  float* ck = nullptr;           // cap_ck states: the state before outer c * m
  float* seg = nullptr;          // cap_seg states: the states of one recomputed segment
  float* ubar = nullptr;         // tape: K x H x W
  uint8_t* M = nullptr;          // tape: K x (n1 + n2) projection pass bits
  float *Ph = nullptr, *Pb = nullptr;  // phat / pbar (n1 + n2 each) when the handle has none
  float *Au = nullptr, *Ad = nullptr, *Af = nullptr;
  double* Aal = nullptr;
  float *AP = nullptr, *AQ = nullptr, *APh = nullptr;  // n1 + n2 each
  float *AL = nullptr, *APp = nullptr;                 // nh + nv, 2 (nh + nv)
  int4 *rowtab = nullptr, *coltab = nullptr;           // H, W: tile index, first, end
  bool fused = false;   // the tile-fused reverse kernel applies
  float* tapeF = nullptr;  // its tape
  int nal = 0;          // alpha partial-sum slots
  // one graph per segment (recompute + reverse of its outer iterations), valid for
  // the (N, m, mask) they were captured with
  std::vector<cudaGraphExec_t> graphs;
  int g_N = -1, g_m = -1;
  const uint8_t* g_mask = nullptr;
};

struct dd_tv {
  dd_tv_params p;
  Grid g;            // decomposition grid (1 x 1 for the full-dimension path)
  int fid;
  cudaStream_t stream = nullptr;   // where work is issued: the caller's stream or `own`
  cudaStream_t own = nullptr;      // private blocking stream (orders with the legacy stream)
  int device = 0;
  char err[512] = {0};
  int n = 0;         // outer iterations since load / set_state
  bool loaded = false;
  bool has_mask = false;

  size_t npx = 0, n1 = 0, n2 = 0, nh = 0, nv = 0;
  float *f = nullptr, *u = nullptr, *P1 = nullptr, *P2 = nullptr, *lamh = nullptr, *lamv = nullptr;
  uint8_t* mask = nullptr;
  float* strip_mem = nullptr;
  Strips strips[2] = {};   // every interface line of the handle (the multiplier update's view)
  // The local solves' view of the horizontal lines: for a row-block shard whose top
  // side is cut, line -1 (the cut above) precedes line 0 in memory, so these point one
  // line into the arrays above; for a whole image they equal lamh / strips.
  float* lamh_k = nullptr;
  Strips strips_k[2] = {};
  // row-block shard (dd_tv_create_shard): global tile rows [tile_row0, tile_row0 + g.NR)
  // of a problem with nr_global tile rows; its first pixel row is row0 of the image
  bool shard = false;
  int tile_row0 = 0, nr_global = 0, row0 = 0;
  size_t nlh = 0;          // horizontal interface lines held, cut lines included
  Coef* coef = nullptr;
  // plain path: phat and pbar; full-dimension path: pbar (carried across iterations)
  float *Ph1 = nullptr, *Ph2 = nullptr, *Pb1 = nullptr, *Pb2 = nullptr;
  double* partials = nullptr;
  unsigned int* counter = nullptr;
  double* red_out = nullptr;
  int* flag = nullptr;
  int* inner_used = nullptr;             // NR * NC (adaptive inner stopping)
  int* inner_max = nullptr;              // 1
  unsigned long long* inner_work = nullptr;  // 1

  cudaGraphExec_t chunk[2] = {nullptr, nullptr};  // kGraphChunk outer iterations from parity 0 / 1
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;

  // measurement hooks: event pairs bracketing each phase while profiling is on
  struct Mark {
    cudaEvent_t a, b;
    int slot;
  };
  bool prof = false;
  std::vector<Mark> marks;
  long long prof_launches[3] = {0, 0, 0};

  long long gen = 0;             // incremented by every load (invalidates checkpoints)
  AdjointWork* adj = nullptr;
};

namespace {

int fail(dd_tv* h, int code, const char* fmt, ...) {
  if (h) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(h->err, sizeof(h->err), fmt, ap);
    va_end(ap);
  }
  return code;
}

// a shard exchanges its cut strips with its neighbours between outer iterations, so
// the calls that run several outer iterations or read the global state refuse it
int refuse_shard(dd_tv* h, const char* what) {
  return fail(h, DD_TV_EUNSUPPORTED, "%s is not available on a shard (one outer iteration per dd_tv_iterate call, "
              "with dd_tv_shard_export / dd_tv_shard_import between calls)", what);
}

#define CK(call)                                                                                  \
  do {                                                                                            \
    cudaError_t e_ = (call);                                                                      \
    if (e_ != cudaSuccess) return fail(h, DD_TV_ECUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
  } while (0)

template <class T>
int dalloc(dd_tv* h, T** ptr, size_t count) {
  *ptr = nullptr;
  if (count == 0) return DD_TV_OK;
  cudaError_t e = cudaMalloc((void**)ptr, count * sizeof(T));
  if (e != cudaSuccess) {
    *ptr = nullptr;
    return fail(h, DD_TV_ENOMEM, "cudaMalloc(%zu bytes): %s", count * sizeof(T), cudaGetErrorString(e));
  }
  return DD_TV_OK;
}

int validate(const dd_tv_params* p, char* msg, size_t len) {
#define BAD(...) (snprintf(msg, len, __VA_ARGS__), DD_TV_EINVAL)
  if (!p) return BAD("params is NULL");
  if (p->height < 1 || p->width < 1) return BAD("height and width must be >= 1 (got %d x %d)", p->height, p->width);
  if ((long long)p->height * p->width > (1LL << 31) - 1) return BAD("image larger than 2^31 - 1 pixels");
  if (p->path < DD_TV_PATH_FUSED || p->path > DD_TV_PATH_FULLDIM) return BAD("unknown path %d", p->path);
  if (p->path != DD_TV_PATH_FULLDIM) {
    if (p->sub_rows < 1 || p->sub_rows > p->height) return BAD("sub_rows must be in [1, height] (got %d)", p->sub_rows);
    if (p->sub_cols < 1 || p->sub_cols > p->width) return BAD("sub_cols must be in [1, width] (got %d)", p->sub_cols);
    // the interface kernels number the edges in 32-bit integers
    const long long edges = (long long)(p->sub_rows - 1) * p->width + (long long)(p->sub_cols - 1) * p->height;
    if (edges > (1LL << 30) - 1) return BAD("too many interface edges (%lld > 2^30 - 1): use fewer subdomains", edges);
  }
  if (p->fidelity < DD_TV_L2 || p->fidelity > DD_TV_SEG) return BAD("unknown fidelity %d", p->fidelity);
  if (!(p->alpha > 0.0) || !std::isfinite(p->alpha)) return BAD("alpha must be finite and > 0");
  if (p->fidelity == DD_TV_SEG && !(std::isfinite(p->c1) && std::isfinite(p->c2))) return BAD("c1, c2 must be finite");
  if (p->outer_iters < 0) return BAD("outer_iters must be >= 0");
  if (p->inner_iters < 1 || p->inner_iters > DD_TV_MAX_INNER)
    return BAD("inner_iters must be in [1, %d] (got %d)", DD_TV_MAX_INNER, p->inner_iters);
  if (!(p->tau0 > 0.0) || !(p->sigma0 > 0.0) || !std::isfinite(p->tau0) || !std::isfinite(p->sigma0))
    return BAD("tau0 and sigma0 must be finite and > 0");
  // ||div||^2 <= 8 on the pixel grid: tau0 sigma0 ||div||^2 <= 1
  if (p->tau0 * p->sigma0 > 0.125 * (1.0 + 1e-12)) return BAD("tau0 * sigma0 must be <= 1/8");
  if (p->path != DD_TV_PATH_FULLDIM) {
    if (!(p->tau > 0.0) || !(p->sigma > 0.0) || !std::isfinite(p->tau) || !std::isfinite(p->sigma))
      return BAD("tau and sigma must be finite and > 0");
    // ||B||^2 = 2: tau sigma ||B||^2 <= 1 (Algorithm 1 asks tau sigma < 1/2; Section 5 uses 1/2)
    if (p->tau * p->sigma > 0.5 * (1.0 + 1e-12)) return BAD("tau * sigma must be <= 1/2");
    if (!(p->gamma > 0.0) || p->gamma > 1.0 / p->tau * (1.0 + 1e-12))
      return BAD("gamma must be in (0, 1/tau]: the local G^* is only (1/tau)-uniformly convex");
  }
  if (p->path == DD_TV_PATH_FUSED && (p->variant < 0 || p->variant >= fused_num_variants()))
    return BAD("variant must be in [0, %d)", fused_num_variants());
  if (p->outer_tol < 0.0 || !std::isfinite(p->outer_tol)) return BAD("outer_tol must be finite and >= 0");
  if (p->inner_tol < 0.0 || !std::isfinite(p->inner_tol)) return BAD("inner_tol must be finite and >= 0");
  if (p->outer_tol > 0.0) {
    if (!std::isfinite(p->energy_ref) || p->energy_ref == 0.0) return BAD("outer_tol needs a finite nonzero energy_ref");
    if (p->energy_every < 1) return BAD("outer_tol needs energy_every >= 1");
  }
  return DD_TV_OK;
#undef BAD
}

void build_schedule(const dd_tv_params& p, std::vector<Coef>& c) {
  const int K = p.inner_iters;
  c.resize(K);
  const double a = p.alpha;
  if (p.path == DD_TV_PATH_FULLDIM) {
    // plain primal-dual iteration: constant steps, theta = 1, no proximal term
    const double s = p.sigma0, t = p.tau0;
    for (int k = 0; k < K; ++k)
      c[k] = Coef{(float)s, (float)(1.0 / (1.0 + s * a)), (float)(s * a / (1.0 + s * a)), (float)(s * a), 1.0f,
                  (float)t, 0.0f, 1.0f};
    return;
  }
  // accelerated local iteration, restarted at every outer iteration
  double tk = p.tau0, sk = p.sigma0;
  const double tau = p.tau;
  for (int k = 0; k < K; ++k) {
    const double th = 1.0 / std::sqrt(1.0 + 2.0 * p.gamma * tk);
    c[k] = Coef{(float)sk,
                (float)(1.0 / (1.0 + sk * a)),
                (float)(sk * a / (1.0 + sk * a)),
                (float)(sk * a),
                (float)(tau / (tau + tk)),
                (float)(tau * tk / (tau + tk)),
                (float)(tk / (tau + tk)),
                (float)th};
    tk = th * tk;
    sk = sk / th;
  }
}

LocalArgs local_args(dd_tv* h, int write_set) {
  LocalArgs a;
  a.g = h->g;
  a.K = h->p.inner_iters;
  a.tau = (float)h->p.tau;
  a.c1 = (float)h->p.c1;
  a.c2 = (float)h->p.c2;
  a.f = h->f;
  a.mask = h->has_mask ? h->mask : nullptr;
  a.u = h->u;
  a.P1 = h->P1;
  a.P2 = h->P2;
  a.lamh = h->lamh_k;
  a.lamv = h->lamv;
  a.out = h->strips_k[write_set];
  a.coef = h->coef;
  a.err = h->flag;
  a.inner_tol2 = h->p.inner_tol * h->p.inner_tol;
  a.inner_used = h->inner_used;
  a.inner_max = h->inner_max;
  a.inner_work = h->inner_work;
  return a;
}

// Phase brackets for the measurement hooks (no-ops unless profiling is on).
struct PhaseMark {
  dd_tv* h;
  int slot;
  cudaEvent_t a = nullptr;
  PhaseMark(dd_tv* h_, int slot_, int launches) : h(h_), slot(slot_) {
    if (!h->prof) return;
    h->prof_launches[slot] += launches;
    if (cudaEventCreate(&a) == cudaSuccess) cudaEventRecord(a, h->stream);
  }
  ~PhaseMark() {
    if (!h->prof || !a) return;
    cudaEvent_t b = nullptr;
    if (cudaEventCreate(&b) == cudaSuccess) {
      cudaEventRecord(b, h->stream);
      h->marks.push_back(dd_tv::Mark{a, b, slot});
    } else {
      cudaEventDestroy(a);
    }
  }
};

// One outer iteration starting from parity `par` (= n mod 2): the strips of p~^n are
// in set par, those of p~^{n-1} in set 1 - par, and p~^{n+1}'s go to set 1 - par.
cudaError_t outer_once(dd_tv* h, int par) {
  cudaError_t e;
  const cudaStream_t st = h->stream;
  if (h->p.path == DD_TV_PATH_FULLDIM) {
    LocalArgs a = local_args(h, 0);
    PhaseMark m(h, 1, 2 * a.K);
    for (int k = 0; k < a.K; ++k) {
      if ((e = launch_plain_ustep(a, h->Pb1, h->Pb2, h->coef + k, h->fid, st)) != cudaSuccess) return e;
      if ((e = launch_plain_pstep(a, nullptr, nullptr, h->Pb1, h->Pb2, h->coef + k, false, st)) != cudaSuccess)
        return e;
    }
    return cudaSuccess;
  }
  {
    PhaseMark m(h, 0, (h->nh + h->nv) ? 1 : 0);
    // the multiplier update runs over every line the handle holds (a shard's cut lines
    // included): a grid with nlh + 1 tile rows has nlh horizontal interface lines
    Grid gi = h->g;
    gi.NR = (int)h->nlh + 1;
    if ((e = launch_interface(gi, (float)h->p.sigma, h->strips[par], h->strips[1 - par], h->lamh, h->lamv, st)) !=
        cudaSuccess)
      return e;
  }
  LocalArgs a = local_args(h, 1 - par);
  if (h->p.path == DD_TV_PATH_FUSED) {
    PhaseMark m(h, 1, 1);
    return launch_fused_local(a, h->fid, h->p.variant, st);
  }
  PhaseMark m(h, 1, 1 + 2 * a.K + ((h->nh + h->nv) ? 1 : 0));
  if ((e = launch_plain_phat(a, h->Ph1, h->Ph2, h->Pb1, h->Pb2, st)) != cudaSuccess) return e;
  for (int k = 0; k < a.K; ++k) {
    if ((e = launch_plain_ustep(a, h->Pb1, h->Pb2, h->coef + k, h->fid, st)) != cudaSuccess) return e;
    if ((e = launch_plain_pstep(a, h->Ph1, h->Ph2, h->Pb1, h->Pb2, h->coef + k, k + 1 == a.K, st)) != cudaSuccess)
      return e;
  }
  return cudaSuccess;
}

void drop_graphs(dd_tv* h) {
  for (auto& g : h->chunk)
    if (g) {
      cudaGraphExecDestroy(g);
      g = nullptr;
    }
}

int capture_chunk(dd_tv* h, int par) {
  cudaGraph_t graph = nullptr;
  CK(cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal));
  cudaError_t e = cudaSuccess;
  for (int q = 0; q < kGraphChunk && e == cudaSuccess; ++q) e = outer_once(h, (par + q) & 1);
  cudaError_t e2 = cudaStreamEndCapture(h->stream, &graph);
  if (e != cudaSuccess || e2 != cudaSuccess) {
    if (graph) cudaGraphDestroy(graph);
    return fail(h, DD_TV_ECUDA, "graph capture failed: %s",
                cudaGetErrorString(e != cudaSuccess ? e : e2));
  }
  e = cudaGraphInstantiate(&h->chunk[par], graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) {
    h->chunk[par] = nullptr;
    return fail(h, DD_TV_ECUDA, "cudaGraphInstantiate: %s", cudaGetErrorString(e));
  }
  return DD_TV_OK;
}

int run_outer(dd_tv* h, int count) {
  int done = 0;
  while (done < count) {
    const int par = h->n & 1;
    if (count - done >= kGraphChunk && !h->prof) {
      if (!h->chunk[par]) {
        int rc = capture_chunk(h, par);
        if (rc) return rc;
      }
      CK(cudaGraphLaunch(h->chunk[par], h->stream));
      h->n += kGraphChunk;
      done += kGraphChunk;
    } else {
      CK(outer_once(h, par));
      h->n += 1;
      done += 1;
    }
  }
  return DD_TV_OK;
}

int reset_state(dd_tv* h) {
  const cudaStream_t st = h->stream;
  CK(launch_init_u(h->g, h->fid, h->f, h->has_mask ? h->mask : nullptr, h->u, st));
  CK(cudaMemsetAsync(h->P1, 0, h->n1 * sizeof(float), st));
  CK(cudaMemsetAsync(h->P2, 0, h->n2 * sizeof(float), st));
  if (h->nh) CK(cudaMemsetAsync(h->lamh, 0, h->nh * sizeof(float), st));
  if (h->nv) CK(cudaMemsetAsync(h->lamv, 0, h->nv * sizeof(float), st));
  if (h->strip_mem) CK(cudaMemsetAsync(h->strip_mem, 0, 4 * (h->nh + h->nv) * sizeof(float), st));
  if (h->Pb1) {
    CK(cudaMemsetAsync(h->Pb1, 0, h->n1 * sizeof(float), st));
    CK(cudaMemsetAsync(h->Pb2, 0, h->n2 * sizeof(float), st));
  }
  CK(cudaMemsetAsync(h->inner_used, 0, (size_t)h->g.NR * h->g.NC * sizeof(int), st));
  CK(cudaMemsetAsync(h->inner_max, 0, sizeof(int), st));
  CK(cudaMemsetAsync(h->inner_work, 0, sizeof(unsigned long long), st));
  h->n = 0;
  h->loaded = true;
  return DD_TV_OK;
}

// Reads (and clears) the device flag a kernel sets when a bounded wait ran out.
int check_timeout(dd_tv* h) {
  int v = 0;
  CK(cudaMemcpyAsync(&v, h->flag, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  if (v) {
    CK(cudaMemsetAsync(h->flag, 0, sizeof(int), h->stream));
    return fail(h, DD_TV_ETIMEOUT, "a device-side wait of the fused kernel ran out (results are invalid)");
  }
  return DD_TV_OK;
}

int energy_of(dd_tv* h, const float* u, const float* f, const uint8_t* mask, bool dual, double* out2) {
  {
    PhaseMark m(h, 2, 1);
    CK(launch_energy(h->g, h->fid, (float)h->p.alpha, (float)h->p.c1, (float)h->p.c2, u, f, mask,
                   dual ? h->P1 : nullptr, dual ? h->P2 : nullptr, h->partials, h->counter, h->red_out, h->stream));
  }
  CK(cudaMemcpyAsync(out2, h->red_out, 2 * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  return DD_TV_OK;
}

int solve_loaded(dd_tv* h, dd_tv_stats* stats, bool sync_needed) {
  const dd_tv_params& p = h->p;
  const bool tol = p.outer_tol > 0.0;
  if (stats) {
    stats->outer_done = 0;
    stats->pixel_iters = 0;
    stats->energy = NAN;
    stats->rel_err = NAN;
    stats->ms = NAN;
    stats->converged = 0;
  }
  const bool adaptive = p.inner_tol > 0.0;
  if (adaptive) {
    CK(cudaMemsetAsync(h->inner_max, 0, sizeof(int), h->stream));
    CK(cudaMemsetAsync(h->inner_work, 0, sizeof(unsigned long long), h->stream));
  }
  CK(cudaEventRecord(h->ev0, h->stream));
  int done = 0, rc;
  bool conv = false;
  double J = NAN;
  if (!tol) {
    if ((rc = run_outer(h, p.outer_iters))) return rc;
    done = p.outer_iters;
  } else {
    while (done < p.outer_iters && !conv) {
      const int step = std::min(p.energy_every, p.outer_iters - done);
      if ((rc = run_outer(h, step))) return rc;
      done += step;
      double o[2];
      if ((rc = energy_of(h, h->u, h->f, h->has_mask ? h->mask : nullptr, false, o))) return rc;
      J = o[0];
      conv = (J - p.energy_ref) / std::fabs(p.energy_ref) <= p.outer_tol;
    }
  }
  CK(cudaEventRecord(h->ev1, h->stream));
  if (stats || sync_needed) {
    CK(cudaEventSynchronize(h->ev1));
    if ((rc = check_timeout(h))) return rc;
  }
  CK(cudaGetLastError());
  if (stats) {
    float ms = 0.f;
    CK(cudaEventElapsedTime(&ms, h->ev0, h->ev1));
    stats->outer_done = done;
    stats->pixel_iters = (long long)p.height * p.width * p.inner_iters * (long long)done;
    stats->inner_max = done > 0 ? p.inner_iters : 0;
    if (adaptive) {
      int mx = 0;
      unsigned long long work = 0;
      CK(cudaMemcpyAsync(&mx, h->inner_max, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
      CK(cudaMemcpyAsync(&work, h->inner_work, sizeof(work), cudaMemcpyDeviceToHost, h->stream));
      CK(cudaStreamSynchronize(h->stream));
      stats->inner_max = mx;
      stats->pixel_iters = (long long)work;
    }
    stats->energy = J;
    stats->rel_err = std::isnan(J) ? NAN : (J - p.energy_ref) / std::fabs(p.energy_ref);
    stats->ms = ms;
    stats->converged = conv ? 1 : 0;
  }
  if (tol && !conv) return fail(h, DD_TV_ENOTCONV, "outer_tol %.3g not reached in %d outer iterations", p.outer_tol, done);
  return DD_TV_OK;
}

int load_common(dd_tv* h, const float* f, const uint8_t* mask, cudaMemcpyKind kind) {
  if (!h) return DD_TV_EINVAL;
  if (!f) return fail(h, DD_TV_EINVAL, "f is NULL");
  if (mask && h->fid == DD_TV_SEG) return fail(h, DD_TV_EINVAL, "an inpainting mask is not defined for DD_TV_SEG");
  CK(cudaMemcpyAsync(h->f, f, h->npx * sizeof(float), kind, h->stream));
  h->has_mask = mask != nullptr;
  if (mask) {
    if (!h->mask) {
      int rc = dalloc(h, &h->mask, h->npx);
      if (rc) return rc;
      drop_graphs(h);
    }
    CK(cudaMemcpyAsync(h->mask, mask, h->npx, kind, h->stream));
  }
  drop_graphs(h);  // the mask pointer captured in the graphs may have changed
  ++h->gen;
  return reset_state(h);
}

// ---- reverse pass of the unrolled outer iterations (dd_tv_adjoint_*)

void adj_drop_graphs(AdjointWork* w) {
  for (auto& g : w->graphs)
    if (g) cudaGraphExecDestroy(g);
  w->graphs.clear();
  w->g_N = w->g_m = -1;
}

void adj_free(AdjointWork* w) {
  if (!w) return;
  adj_drop_graphs(w);
  void* bufs[] = {w->ck, w->seg, w->ubar, w->M, w->Ph, w->Pb, w->Au, w->Ad, w->Af, w->Aal, w->AP, w->AQ, w->APh,
                  w->AL, w->APp, w->rowtab, w->coltab, w->tapeF};
  for (void* b : bufs)
    if (b) cudaFree(b);
  delete w;
}

// Allocates the fixed part of the workspace once per handle and grows the saved-state
// slots to nck checkpoints and m segment states.
int adj_reserve(dd_tv* h, int nck, int m) {
  if (!h->adj) {
    if (std::max(adj_alpha_slots(h->g), adj_alpha_slots_fused(h->g)) > (1LL << 30))
      return fail(h, DD_TV_EUNSUPPORTED, "too many subdomains for the reverse pass");
    AdjointWork* w = new (std::nothrow) AdjointWork();
    if (!w) return fail(h, DD_TV_ENOMEM, "out of host memory");
    h->adj = w;
    const size_t K = (size_t)h->p.inner_iters, nP = h->n1 + h->n2, ne = h->nh + h->nv;
    w->slot = h->npx + nP + 5 * ne;
    const size_t tape_f = adj_fused_tape_floats(h->g, h->p.inner_iters);
    // the fused reverse kernel keeps a per-CTA tape; beyond 4 GiB use the per-step path
    w->fused = tape_f > 0 && tape_f * sizeof(float) <= (4ull << 30);
    w->nal = (int)std::max(adj_alpha_slots(h->g), adj_alpha_slots_fused(h->g));
    if (w->fused) CK(adj_fused_prepare());
    int rc;
    if ((rc = dalloc(h, &w->Au, h->npx)) || (rc = dalloc(h, &w->Ad, h->npx)) || (rc = dalloc(h, &w->Af, h->npx)) ||
        (rc = dalloc(h, &w->Aal, (size_t)w->nal)) || (rc = dalloc(h, &w->AP, nP)) || (rc = dalloc(h, &w->AQ, nP)) ||
        (rc = dalloc(h, &w->APh, nP)) || (rc = dalloc(h, &w->AL, ne)) || (rc = dalloc(h, &w->APp, 2 * ne))) {
      adj_free(w);
      h->adj = nullptr;
      return rc;
    }
    if (w->fused) {
      if ((rc = dalloc(h, &w->tapeF, tape_f))) {
        adj_free(w);
        h->adj = nullptr;
        return rc;
      }
    } else {
      // per-step reverse: the tape in global memory, the plain path's phat / pbar, and
      // the tile tables of the per-pixel kernels
      if ((rc = dalloc(h, &w->ubar, K * h->npx)) || (rc = dalloc(h, &w->M, K * nP)) ||
          (rc = dalloc(h, &w->rowtab, h->g.H)) || (rc = dalloc(h, &w->coltab, h->g.W)) ||
          (!h->Ph1 && ((rc = dalloc(h, &w->Ph, nP)) || (rc = dalloc(h, &w->Pb, nP))))) {
        adj_free(w);
        h->adj = nullptr;
        return rc;
      }
      // inactive dofs are never written by the tape: their pass bits stay 0
      CK(cudaMemsetAsync(w->M, 0, K * nP, h->stream));
      std::vector<int4> rt(h->g.H), ct(h->g.W);
      for (int a = 0; a < h->g.NR; ++a)
        for (int i = part_start(a, h->g.H, h->g.NR); i < part_start(a + 1, h->g.H, h->g.NR); ++i)
          rt[i] = make_int4(a, part_start(a, h->g.H, h->g.NR), part_start(a + 1, h->g.H, h->g.NR), 0);
      for (int b = 0; b < h->g.NC; ++b)
        for (int j = part_start(b, h->g.W, h->g.NC); j < part_start(b + 1, h->g.W, h->g.NC); ++j)
          ct[j] = make_int4(b, part_start(b, h->g.W, h->g.NC), part_start(b + 1, h->g.W, h->g.NC), 0);
      CK(cudaMemcpy(w->rowtab, rt.data(), rt.size() * sizeof(int4), cudaMemcpyHostToDevice));
      CK(cudaMemcpy(w->coltab, ct.data(), ct.size() * sizeof(int4), cudaMemcpyHostToDevice));
    }
  }
  AdjointWork* w = h->adj;
  if (nck > w->cap_ck || m > w->cap_seg) adj_drop_graphs(w);  // they hold the slot addresses
  if (nck > w->cap_ck) {
    if (w->ck) cudaFree(w->ck);
    w->ck = nullptr;
    w->cap_ck = 0;
    int rc = dalloc(h, &w->ck, (size_t)nck * w->slot);
    if (rc) return rc;
    w->cap_ck = nck;
  }
  if (m > w->cap_seg) {
    if (w->seg) cudaFree(w->seg);
    w->seg = nullptr;
    w->cap_seg = 0;
    int rc = dalloc(h, &w->seg, (size_t)m * w->slot);
    if (rc) return rc;
    w->cap_seg = m;
  }
  return DD_TV_OK;
}

// saved state: [u | P1 | P2 | lamh | lamv | both strip sets]
int state_save(dd_tv* h, float* dst) {
  const cudaStream_t st = h->stream;
  const auto D2D = cudaMemcpyDeviceToDevice;
  const size_t ne = h->nh + h->nv;
  CK(cudaMemcpyAsync(dst, h->u, h->npx * sizeof(float), D2D, st));
  dst += h->npx;
  CK(cudaMemcpyAsync(dst, h->P1, h->n1 * sizeof(float), D2D, st));
  dst += h->n1;
  CK(cudaMemcpyAsync(dst, h->P2, h->n2 * sizeof(float), D2D, st));
  dst += h->n2;
  if (ne) {
    if (h->nh) CK(cudaMemcpyAsync(dst, h->lamh, h->nh * sizeof(float), D2D, st));
    if (h->nv) CK(cudaMemcpyAsync(dst + h->nh, h->lamv, h->nv * sizeof(float), D2D, st));
    CK(cudaMemcpyAsync(dst + ne, h->strip_mem, 4 * ne * sizeof(float), D2D, st));
  }
  return DD_TV_OK;
}

int state_restore(dd_tv* h, const float* src, int n) {
  const cudaStream_t st = h->stream;
  const auto D2D = cudaMemcpyDeviceToDevice;
  const size_t ne = h->nh + h->nv;
  CK(cudaMemcpyAsync(h->u, src, h->npx * sizeof(float), D2D, st));
  src += h->npx;
  CK(cudaMemcpyAsync(h->P1, src, h->n1 * sizeof(float), D2D, st));
  src += h->n1;
  CK(cudaMemcpyAsync(h->P2, src, h->n2 * sizeof(float), D2D, st));
  src += h->n2;
  if (ne) {
    if (h->nh) CK(cudaMemcpyAsync(h->lamh, src, h->nh * sizeof(float), D2D, st));
    if (h->nv) CK(cudaMemcpyAsync(h->lamv, src + h->nh, h->nv * sizeof(float), D2D, st));
    CK(cudaMemcpyAsync(h->strip_mem, src + ne, 4 * ne * sizeof(float), D2D, st));
  }
  h->n = n;
  return DD_TV_OK;
}

AdjArgs adj_args(dd_tv* h) {
  AdjointWork* w = h->adj;
  AdjArgs r;
  r.g = h->g;
  r.fid = h->fid;
  r.c1 = (float)h->p.c1;
  r.c2 = (float)h->p.c2;
  r.f = h->f;
  r.mask = h->has_mask ? h->mask : nullptr;
  r.Au = w->Au;
  r.Ad = w->Ad;
  r.Af = w->Af;
  r.Aal = w->Aal;
  r.AP1 = w->AP;
  r.AP2 = w->AP + h->n1;
  r.AQ1 = w->AQ;
  r.AQ2 = w->AQ + h->n1;
  r.APh1 = w->APh;
  r.APh2 = w->APh + h->n1;
  r.ALh = w->AL;
  r.ALv = w->AL + h->nh;
  r.APp = Strips{w->APp, w->APp + h->nh, w->APp + 2 * h->nh, w->APp + 2 * h->nh + h->nv};
  r.rowtab = w->rowtab;
  r.coltab = w->coltab;
  r.tape = w->tapeF;
  return r;
}

// Recomputes outer iteration n from the state in the handle's buffers (h->n = n) and
// runs the reverse of its local solves: in one tile-fused kernel (tape in shared
// memory) when the tile shape and K allow, else with the plain path's kernels
// recording the tape in global memory followed by the global-memory reverse kernels.
int reverse_outer(dd_tv* h, const AdjArgs& r);

int tape_outer(dd_tv* h, const AdjArgs& r) {
  AdjointWork* w = h->adj;
  const cudaStream_t st = h->stream;
  const int par = h->n & 1;
  CK(launch_interface(h->g, (float)h->p.sigma, h->strips[par], h->strips[1 - par], h->lamh, h->lamv, st));
  LocalArgs a = local_args(h, 1 - par);
  if (w->fused) {
    CK(launch_adj_fused(a, r, h->fid, st));
    CK(launch_adj_interface(r, (float)h->p.sigma, (float)h->p.tau, st));
    return DD_TV_OK;
  }
  const size_t nP = h->n1 + h->n2;
  float* Ph1 = h->Ph1 ? h->Ph1 : w->Ph;
  float* Ph2 = h->Ph1 ? h->Ph2 : w->Ph + h->n1;
  float* Pb1 = h->Ph1 ? h->Pb1 : w->Pb;
  float* Pb2 = h->Ph1 ? h->Pb2 : w->Pb + h->n1;
  CK(launch_plain_phat(a, Ph1, Ph2, Pb1, Pb2, st));
  for (int k = 0; k < a.K; ++k) {
    uint8_t* Mk = w->M + (size_t)k * nP;
    CK(launch_ustep_tape(a, w->rowtab, w->coltab, Pb1, Pb2, h->coef + k, h->fid, w->ubar + (size_t)k * h->npx, st));
    CK(launch_pstep_tape(a, w->rowtab, w->coltab, Ph1, Ph2, Pb1, Pb2, h->coef + k, Mk, Mk + h->n1, st));
  }
  return reverse_outer(h, r);
}

// Reverse of outer iteration n from the tape in global memory (after tape_outer).
int reverse_outer(dd_tv* h, const AdjArgs& r) {
  AdjointWork* w = h->adj;
  const cudaStream_t st = h->stream;
  const int K = h->p.inner_iters;
  const size_t nP = h->n1 + h->n2;
  for (int k = K - 1; k >= 0; --k) {
    const uint8_t* Mk = w->M + (size_t)k * nP;
    CK(launch_adj_inner(r, h->coef + k, w->ubar + (size_t)k * h->npx, Mk, Mk + h->n1, k == K - 1, k == 0, st));
  }
  CK(launch_adj_interface(r, (float)h->p.sigma, (float)h->p.tau, st));
  return DD_TV_OK;
}

// Recompute segment c from its checkpoint and run the reverse of its outer iterations.
int adj_segment(dd_tv* h, const AdjArgs& r, int c) {
  AdjointWork* w = h->adj;
  const int s0 = c * w->m, e0 = std::min(s0 + w->m, w->N);
  int rc;
  if ((rc = state_restore(h, w->ck + (size_t)c * w->slot, s0))) return rc;
  for (int n = s0; n < e0; ++n) {
    if ((rc = state_save(h, w->seg + (size_t)(n - s0) * w->slot))) return rc;
    if (n + 1 < e0) {
      CK(outer_once(h, n & 1));
      h->n = n + 1;
    }
  }
  for (int n = e0 - 1; n >= s0; --n) {
    if ((rc = state_restore(h, w->seg + (size_t)(n - s0) * w->slot, n))) return rc;
    if ((rc = tape_outer(h, r))) return rc;
  }
  return DD_TV_OK;
}

int adj_capture_segment(dd_tv* h, const AdjArgs& r, int c, cudaGraphExec_t* out) {
  cudaGraph_t graph = nullptr;
  CK(cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal));
  const int rc = adj_segment(h, r, c);
  const cudaError_t e2 = cudaStreamEndCapture(h->stream, &graph);
  if (rc || e2 != cudaSuccess) {
    if (graph) cudaGraphDestroy(graph);
    return rc ? rc : fail(h, DD_TV_ECUDA, "adjoint graph capture failed: %s", cudaGetErrorString(e2));
  }
  const cudaError_t e = cudaGraphInstantiate(out, graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) {
    *out = nullptr;
    return fail(h, DD_TV_ECUDA, "cudaGraphInstantiate: %s", cudaGetErrorString(e));
  }
  return DD_TV_OK;
}

}  // namespace

extern "C" {

void dd_tv_default_params(dd_tv_params* p) {
  if (!p) return;
  std::memset(p, 0, sizeof(*p));
  p->height = p->width = 1;
  p->sub_rows = p->sub_cols = 1;
  p->fidelity = DD_TV_L2;
  p->alpha = 10.0;
  p->outer_iters = 100;
  p->inner_iters = 10;
  p->tau = 50.0;
  p->sigma = 1.0 / (2.0 * 50.0);
  p->tau0 = 10.0;
  p->sigma0 = 1.0 / 80.0;
  p->gamma = 1.0 / (8.0 * 50.0);
  p->outer_tol = 0.0;
  p->energy_ref = NAN;
  p->energy_every = 5;
  p->path = DD_TV_PATH_FUSED;
  p->inner_tol = 0.0;
}

namespace {

// a0 < 0: the whole image; otherwise the row-block shard of tile rows [a0, a1)
int create_impl(dd_tv** out, const dd_tv_params* p, int a0, int a1) {
  if (!out) return DD_TV_EINVAL;
  *out = nullptr;
  dd_tv* h = new (std::nothrow) dd_tv();
  if (!h) return DD_TV_ENOMEM;
  int rc = validate(p, h->err, sizeof(h->err));
  if (!rc && a0 >= 0) {
    if (p->path != DD_TV_PATH_FUSED) {
      fail(h, DD_TV_EUNSUPPORTED, "a shard runs the fused path only");
      rc = DD_TV_EUNSUPPORTED;
    } else if (p->inner_tol > 0.0) {
      fail(h, DD_TV_EUNSUPPORTED, "a shard runs a fixed number of inner iterations (inner_tol must be 0)");
      rc = DD_TV_EUNSUPPORTED;
    } else if (a1 <= a0 || a1 > p->sub_rows) {
      fail(h, DD_TV_EINVAL, "shard tile rows [%d, %d) must be a nonempty range inside [0, %d)", a0, a1, p->sub_rows);
      rc = DD_TV_EINVAL;
    } else if (p->height % p->sub_rows != 0) {
      fail(h, DD_TV_EINVAL, "sharding needs tile rows of equal height: height %d is not a multiple of sub_rows %d",
           p->height, p->sub_rows);
      rc = DD_TV_EINVAL;
    }
  }
  if (rc) {
    std::snprintf(g_create_err, sizeof(g_create_err), "%s", h->err);
    delete h;
    return rc;
  }
  h->p = *p;
  h->fid = p->fidelity;
  const bool full = p->path == DD_TV_PATH_FULLDIM;
  h->g = Grid{p->height, p->width, full ? 1 : p->sub_rows, full ? 1 : p->sub_cols};
  if (a0 >= 0) {
    // the shard's own problem: its rows, with the sides towards other shards cut
    const int th = p->height / p->sub_rows;
    h->shard = true;
    h->tile_row0 = a0;
    h->nr_global = p->sub_rows;
    h->row0 = a0 * th;
    h->g = Grid{(a1 - a0) * th, p->width, a1 - a0, p->sub_cols};
    h->g.cut_top = a0 > 0;
    h->g.cut_bot = a1 < p->sub_rows;
    h->p.height = h->g.H;
    h->p.sub_rows = h->g.NR;
  }
  if (p->inner_tol > 0.0 && p->path != DD_TV_PATH_FUSED) {
    fail(h, DD_TV_EUNSUPPORTED, "inner_tol > 0 (adaptive inner stopping) needs the fused path");
    std::snprintf(g_create_err, sizeof(g_create_err), "%s", h->err);
    delete h;
    return DD_TV_EUNSUPPORTED;
  }
  if (p->path == DD_TV_PATH_FUSED) {
    const int mr = (h->g.H + h->g.NR - 1) / h->g.NR, mc = (h->g.W + h->g.NC - 1) / h->g.NC;
    int maxr, maxc;
    fused_max_tile(&maxr, &maxc);
    if (mr > maxr || mc > maxc) {
      fail(h, DD_TV_EUNSUPPORTED, "fused path supports tiles up to %d x %d (got %d x %d)", maxr, maxc, mr, mc);
      std::snprintf(g_create_err, sizeof(g_create_err), "%s", h->err);
      delete h;
      return DD_TV_EUNSUPPORTED;
    }
  }
  cudaGetDevice(&h->device);
  if (p->path == DD_TV_PATH_FUSED) {
    cudaError_t e = fused_prepare();
    if (e != cudaSuccess) {
      std::snprintf(g_create_err, sizeof(g_create_err), "fused kernel set-up: %s", cudaGetErrorString(e));
      delete h;
      return DD_TV_ECUDA;
    }
  }
  const Grid& g = h->g;
  h->npx = (size_t)g.H * g.W;
  h->n1 = (size_t)(g.H + g.NR) * g.W;
  h->n2 = (size_t)g.H * (g.W + g.NC);
  h->nlh = (size_t)(g.NR - 1) + g.cut_top + g.cut_bot;
  h->nh = h->nlh * g.W;
  h->nv = (size_t)(g.NC - 1) * g.H;
  std::vector<Coef> sched;
  build_schedule(*p, sched);
  if ((rc = dalloc(h, &h->f, h->npx)) || (rc = dalloc(h, &h->u, h->npx)) || (rc = dalloc(h, &h->P1, h->n1)) ||
      (rc = dalloc(h, &h->P2, h->n2)) || (rc = dalloc(h, &h->lamh, h->nh)) || (rc = dalloc(h, &h->lamv, h->nv)) ||
      (rc = dalloc(h, &h->strip_mem, 4 * (h->nh + h->nv))) || (rc = dalloc(h, &h->coef, sched.size())) ||
      (rc = dalloc(h, &h->partials, (size_t)std::max(reduce_partials_count(), sum_f64_partials_count()))) ||
      (rc = dalloc(h, &h->counter, 1)) || (rc = dalloc(h, &h->red_out, 2)) || (rc = dalloc(h, &h->flag, 1)) ||
      (rc = dalloc(h, &h->inner_used, (size_t)h->g.NR * h->g.NC)) || (rc = dalloc(h, &h->inner_max, 1)) ||
      (rc = dalloc(h, &h->inner_work, 1))) {
    std::snprintf(g_create_err, sizeof(g_create_err), "%s", h->err);
    dd_tv_destroy(h);
    return rc;
  }
  if (p->path != DD_TV_PATH_FUSED) {
    if ((rc = dalloc(h, &h->Pb1, h->n1)) || (rc = dalloc(h, &h->Pb2, h->n2))) {
      dd_tv_destroy(h);
      return rc;
    }
  }
  if (p->path == DD_TV_PATH_PLAIN) {
    if ((rc = dalloc(h, &h->Ph1, h->n1)) || (rc = dalloc(h, &h->Ph2, h->n2))) {
      dd_tv_destroy(h);
      return rc;
    }
  }
  // strip sets: [SB | ST | SR | SL] each, both sets in one allocation (float4-aligned
  // when W and H are multiples of 4)
  for (int s = 0; s < 2; ++s) {
    float* base = h->strip_mem ? h->strip_mem + (size_t)s * 2 * (h->nh + h->nv) : nullptr;
    h->strips[s].SB = base;
    h->strips[s].ST = base ? base + h->nh : nullptr;
    h->strips[s].SR = base ? base + 2 * h->nh : nullptr;
    h->strips[s].SL = base ? base + 2 * h->nh + h->nv : nullptr;
    const size_t skip = (size_t)g.cut_top * g.W;  // the cut line above comes first
    h->strips_k[s] = h->strips[s];
    if (base) {
      h->strips_k[s].SB += skip;
      h->strips_k[s].ST += skip;
    }
  }
  h->lamh_k = h->lamh ? h->lamh + (size_t)g.cut_top * g.W : nullptr;
  cudaError_t e;
  if ((e = cudaMemcpy(h->coef, sched.data(), sched.size() * sizeof(Coef), cudaMemcpyHostToDevice)) != cudaSuccess ||
      (e = cudaMemset(h->counter, 0, sizeof(unsigned int))) != cudaSuccess ||
      (e = cudaMemset(h->flag, 0, sizeof(int))) != cudaSuccess ||
      (e = cudaEventCreate(&h->ev0)) != cudaSuccess || (e = cudaEventCreate(&h->ev1)) != cudaSuccess ||
      (e = cudaStreamCreate(&h->own)) != cudaSuccess) {
    std::snprintf(g_create_err, sizeof(g_create_err), "dd_tv_create: %s", cudaGetErrorString(e));
    dd_tv_destroy(h);
    return DD_TV_ECUDA;
  }
  h->stream = h->own;
  *out = h;
  return DD_TV_OK;
}

}  // namespace

int dd_tv_create(dd_tv** out, const dd_tv_params* p) { return create_impl(out, p, -1, -1); }

int dd_tv_create_shard(dd_tv** out, const dd_tv_params* p, int tile_row_begin, int tile_row_end) {
  if (tile_row_begin < 0) {
    if (out) *out = nullptr;
    std::snprintf(g_create_err, sizeof(g_create_err), "shard tile rows must start at 0 or later (got %d)",
                  tile_row_begin);
    return DD_TV_EINVAL;
  }
  return create_impl(out, p, tile_row_begin, tile_row_end);
}

int dd_tv_destroy(dd_tv* h) {
  if (!h) return DD_TV_OK;
  drop_graphs(h);
  adj_free(h->adj);
  h->adj = nullptr;
  for (auto& m : h->marks) {
    cudaEventDestroy(m.a);
    cudaEventDestroy(m.b);
  }
  void* bufs[] = {h->f, h->u, h->P1, h->P2, h->lamh, h->lamv, h->mask, h->strip_mem, h->coef, h->Ph1, h->Ph2,
                  h->Pb1, h->Pb2, h->partials, h->counter, h->red_out, h->flag, h->inner_used, h->inner_max,
                  h->inner_work};
  for (void* b : bufs)
    if (b) cudaFree(b);
  if (h->ev0) cudaEventDestroy(h->ev0);
  if (h->ev1) cudaEventDestroy(h->ev1);
  if (h->own) cudaStreamDestroy(h->own);
  delete h;
  return DD_TV_OK;
}

const char* dd_tv_last_error(const dd_tv* h) {
  if (!h) return g_create_err[0] ? g_create_err : "invalid handle (NULL)";
  return h->err;
}

int dd_tv_set_stream(dd_tv* h, void* stream) {
  if (!h) return DD_TV_EINVAL;
  h->stream = stream ? (cudaStream_t)stream : h->own;
  return DD_TV_OK;
}

int dd_tv_load(dd_tv* h, const float* f_dev, const uint8_t* mask_dev) {
  return load_common(h, f_dev, mask_dev, cudaMemcpyDeviceToDevice);
}

int dd_tv_iterate(dd_tv* h, int n_outer) {
  if (!h) return DD_TV_EINVAL;
  if (!h->loaded) return fail(h, DD_TV_EINVAL, "no data loaded (dd_tv_load or dd_tv_set_state first)");
  if (n_outer < 0) return fail(h, DD_TV_EINVAL, "n_outer must be >= 0");
  if (h->shard && n_outer > 1) return fail(h, DD_TV_EINVAL, "a shard runs one outer iteration per call (got %d)", n_outer);
  return run_outer(h, n_outer);
}

int dd_tv_outer_count(const dd_tv* h) { return h ? h->n : -1; }

int dd_tv_inner_counts(dd_tv* h, int* counts_host, int* max_out) {
  if (!h) return DD_TV_EINVAL;
  if (!counts_host) return fail(h, DD_TV_EINVAL, "counts is NULL");
  const int T = h->g.NR * h->g.NC;
  if (h->p.inner_tol > 0.0) {
    int mx = 0;
    CK(cudaMemcpyAsync(counts_host, h->inner_used, T * sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaMemcpyAsync(&mx, h->inner_max, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaMemsetAsync(h->inner_max, 0, sizeof(int), h->stream));
    CK(cudaStreamSynchronize(h->stream));
    if (max_out) *max_out = mx;
    return DD_TV_OK;
  }
  const int k = h->n > 0 ? h->p.inner_iters : 0;
  for (int t = 0; t < T; ++t) counts_host[t] = k;
  if (max_out) *max_out = k;
  return DD_TV_OK;
}

int dd_tv_get_u(dd_tv* h, float* u_dev) {
  if (!h) return DD_TV_EINVAL;
  if (!u_dev) return fail(h, DD_TV_EINVAL, "u is NULL");
  CK(cudaMemcpyAsync(u_dev, h->u, h->npx * sizeof(float), cudaMemcpyDeviceToDevice, h->stream));
  return DD_TV_OK;
}

int dd_tv_solve(dd_tv* h, const float* f_host, const uint8_t* mask_host, float* u_host, dd_tv_stats* stats) {
  if (!h) return DD_TV_EINVAL;
  if (h->shard) return refuse_shard(h, "dd_tv_solve");
  if (!u_host) return fail(h, DD_TV_EINVAL, "u is NULL");
  int rc = load_common(h, f_host, mask_host, cudaMemcpyHostToDevice);
  if (rc) return rc;
  rc = solve_loaded(h, stats, true);
  if (rc && rc != DD_TV_ENOTCONV) return rc;
  CK(cudaMemcpyAsync(u_host, h->u, h->npx * sizeof(float), cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  return rc;
}

int dd_tv_solve_device(dd_tv* h, const float* f_dev, const uint8_t* mask_dev, float* u_dev, dd_tv_stats* stats) {
  if (!h) return DD_TV_EINVAL;
  if (h->shard) return refuse_shard(h, "dd_tv_solve_device");
  if (!u_dev) return fail(h, DD_TV_EINVAL, "u is NULL");
  int rc = load_common(h, f_dev, mask_dev, cudaMemcpyDeviceToDevice);
  if (rc) return rc;
  rc = solve_loaded(h, stats, false);
  if (rc && rc != DD_TV_ENOTCONV) return rc;
  CK(cudaMemcpyAsync(u_dev, h->u, h->npx * sizeof(float), cudaMemcpyDeviceToDevice, h->stream));
  return rc;
}

int dd_tv_get_state(dd_tv* h, float* u, float* P1, float* P2, float* lamh, float* lamv, float* P1prev,
                    float* P2prev) {
  if (!h) return DD_TV_EINVAL;
  if (h->shard) return refuse_shard(h, "dd_tv_get_state");
  const cudaStream_t st = h->stream;
  const auto D2D = cudaMemcpyDeviceToDevice;
  if (u) CK(cudaMemcpyAsync(u, h->u, h->npx * sizeof(float), D2D, st));
  if (P1) CK(cudaMemcpyAsync(P1, h->P1, h->n1 * sizeof(float), D2D, st));
  if (P2) CK(cudaMemcpyAsync(P2, h->P2, h->n2 * sizeof(float), D2D, st));
  if (lamh && h->nh) CK(cudaMemcpyAsync(lamh, h->lamh, h->nh * sizeof(float), D2D, st));
  if (lamv && h->nv) CK(cudaMemcpyAsync(lamv, h->lamv, h->nv * sizeof(float), D2D, st));
  if (h->p.path == DD_TV_PATH_FULLDIM) {
    if (P1prev) CK(cudaMemcpyAsync(P1prev, h->Pb1, h->n1 * sizeof(float), D2D, st));
    if (P2prev) CK(cudaMemcpyAsync(P2prev, h->Pb2, h->n2 * sizeof(float), D2D, st));
    return DD_TV_OK;
  }
  if (P1prev && P2prev) {
    CK(cudaMemsetAsync(P1prev, 0, h->n1 * sizeof(float), st));
    CK(cudaMemsetAsync(P2prev, 0, h->n2 * sizeof(float), st));
    CK(launch_scatter_strips(h->g, h->strips[1 - (h->n & 1)], P1prev, P2prev, st));
  }
  return DD_TV_OK;
}

int dd_tv_set_state(dd_tv* h, const float* u, const float* P1, const float* P2, const float* lamh,
                    const float* lamv, const float* P1prev, const float* P2prev, int outer_count) {
  if (!h) return DD_TV_EINVAL;
  if (h->shard) return refuse_shard(h, "dd_tv_set_state");
  if (!u || !P1 || !P2) return fail(h, DD_TV_EINVAL, "u, P1 and P2 are required");
  if ((h->nh && !lamh) || (h->nv && !lamv)) return fail(h, DD_TV_EINVAL, "multipliers are required");
  if (!P1prev || !P2prev) return fail(h, DD_TV_EINVAL, "P1prev and P2prev are required");
  if (outer_count < 0) return fail(h, DD_TV_EINVAL, "outer_count must be >= 0");
  const cudaStream_t st = h->stream;
  const auto D2D = cudaMemcpyDeviceToDevice;
  CK(cudaMemcpyAsync(h->u, u, h->npx * sizeof(float), D2D, st));
  CK(cudaMemcpyAsync(h->P1, P1, h->n1 * sizeof(float), D2D, st));
  CK(cudaMemcpyAsync(h->P2, P2, h->n2 * sizeof(float), D2D, st));
  if (h->nh) CK(cudaMemcpyAsync(h->lamh, lamh, h->nh * sizeof(float), D2D, st));
  if (h->nv) CK(cudaMemcpyAsync(h->lamv, lamv, h->nv * sizeof(float), D2D, st));
  h->n = outer_count;
  if (h->p.path == DD_TV_PATH_FULLDIM) {
    CK(cudaMemcpyAsync(h->Pb1, P1prev, h->n1 * sizeof(float), D2D, st));
    CK(cudaMemcpyAsync(h->Pb2, P2prev, h->n2 * sizeof(float), D2D, st));
  } else {
    CK(launch_extract_strips(h->g, P1, P2, h->strips[h->n & 1], st));
    CK(launch_extract_strips(h->g, P1prev, P2prev, h->strips[1 - (h->n & 1)], st));
  }
  h->loaded = true;
  return DD_TV_OK;
}

int dd_tv_energy(dd_tv* h, const float* u_dev, const float* f_dev, const uint8_t* mask_dev, double* J_out) {
  if (!h) return DD_TV_EINVAL;
  if (!u_dev || !f_dev || !J_out) return fail(h, DD_TV_EINVAL, "u, f and J_out are required");
  double o[2];
  int rc = energy_of(h, u_dev, f_dev, mask_dev, false, o);
  if (rc) return rc;
  *J_out = o[0];
  return DD_TV_OK;
}

int dd_tv_gap(dd_tv* h, double* J_out, double* D_out) {
  if (!h) return DD_TV_EINVAL;
  if (h->shard) return refuse_shard(h, "dd_tv_gap");
  if (!h->loaded) return fail(h, DD_TV_EINVAL, "no data loaded");
  const bool dual = h->fid == DD_TV_SEG || (h->fid == DD_TV_L2 && !h->has_mask);
  double o[2];
  int rc = energy_of(h, h->u, h->f, h->has_mask ? h->mask : nullptr, dual, o);
  if (rc) return rc;
  if (J_out) *J_out = o[0];
  if (D_out) *D_out = dual ? o[1] : -INFINITY;
  return DD_TV_OK;
}

int dd_tv_current_energy(dd_tv* h, double* J_out) {
  if (!h) return DD_TV_EINVAL;
  if (!h->loaded) return fail(h, DD_TV_EINVAL, "no data loaded");
  if (!J_out) return fail(h, DD_TV_EINVAL, "J_out is NULL");
  double o[2];
  int rc = energy_of(h, h->u, h->f, h->has_mask ? h->mask : nullptr, false, o);
  if (rc) return rc;
  *J_out = o[0];
  return DD_TV_OK;
}

int dd_tv_set_profiling(dd_tv* h, int on) {
  if (!h) return DD_TV_EINVAL;
  h->prof = on != 0;
  return DD_TV_OK;
}

int dd_tv_set_alpha(dd_tv* h, double alpha) {
  if (!h) return DD_TV_EINVAL;
  dd_tv_params q = h->p;
  q.alpha = alpha;
  char msg[512];
  int rc = validate(&q, msg, sizeof(msg));
  if (rc) return fail(h, rc, "%s", msg);
  std::vector<Coef> sched;
  build_schedule(q, sched);
  // kernels and captured graphs read the schedule from device memory at run time
  CK(cudaStreamSynchronize(h->stream));
  CK(cudaMemcpy(h->coef, sched.data(), sched.size() * sizeof(Coef), cudaMemcpyHostToDevice));
  // checkpoints recorded with the old alpha no longer describe the iteration that a
  // reverse pass would recompute: dd_tv_adjoint_backward needs a new forward
  if (h->adj && alpha != h->p.alpha) h->adj->gen = -1;
  h->p = q;
  return DD_TV_OK;
}

int dd_tv_adjoint_forward(dd_tv* h, const float* f_dev, const uint8_t* mask_dev, int n_outer, int checkpoint_every,
                          float* u_dev) {
  if (!h) return DD_TV_EINVAL;
  if (h->shard) return refuse_shard(h, "dd_tv_adjoint_forward");
  if (h->p.path == DD_TV_PATH_FULLDIM)
    return fail(h, DD_TV_EUNSUPPORTED, "the adjoint is defined for the decomposed paths only");
  if (!u_dev) return fail(h, DD_TV_EINVAL, "u is NULL");
  if (n_outer < 0) return fail(h, DD_TV_EINVAL, "n_outer must be >= 0");
  if (checkpoint_every < 1) return fail(h, DD_TV_EINVAL, "checkpoint_every must be >= 1");
  if (h->p.inner_tol > 0.0)
    return fail(h, DD_TV_EUNSUPPORTED, "the adjoint needs a fixed inner iteration count (inner_tol = 0)");
  int rc = load_common(h, f_dev, mask_dev, cudaMemcpyDeviceToDevice);
  if (rc) return rc;
  const int m = std::max(1, std::min(checkpoint_every, n_outer));
  const int nck = n_outer == 0 ? 0 : (n_outer + m - 1) / m;
  if ((rc = adj_reserve(h, nck, m))) return rc;
  AdjointWork* w = h->adj;
  w->gen = -1;
  for (int c = 0; c < nck; ++c) {
    if ((rc = state_save(h, w->ck + (size_t)c * w->slot))) return rc;
    if ((rc = run_outer(h, std::min(m, n_outer - c * m)))) return rc;
  }
  CK(cudaMemcpyAsync(u_dev, h->u, h->npx * sizeof(float), cudaMemcpyDeviceToDevice, h->stream));
  w->N = n_outer;
  w->m = m;
  w->nck = nck;
  w->gen = h->gen;
  return DD_TV_OK;
}

int dd_tv_adjoint_backward(dd_tv* h, const float* grad_u_dev, float* grad_f_dev, double* grad_alpha) {
  if (!h) return DD_TV_EINVAL;
  if (h->shard) return refuse_shard(h, "dd_tv_adjoint_backward");
  if (!grad_u_dev || !grad_f_dev || !grad_alpha) return fail(h, DD_TV_EINVAL, "grad_u, grad_f and grad_alpha are required");
  AdjointWork* w = h->adj;
  if (!w || w->gen != h->gen) return fail(h, DD_TV_EINVAL, "no dd_tv_adjoint_forward since the last load");
  const cudaStream_t st = h->stream;
  const size_t nP = h->n1 + h->n2, ne = h->nh + h->nv;
  CK(cudaMemcpyAsync(w->Au, grad_u_dev, h->npx * sizeof(float), cudaMemcpyDeviceToDevice, st));
  const int nal = w->nal;
  CK(cudaMemsetAsync(w->Af, 0, h->npx * sizeof(float), st));
  CK(cudaMemsetAsync(w->Aal, 0, nal * sizeof(double), st));
  CK(cudaMemsetAsync(w->AP, 0, nP * sizeof(float), st));
  CK(cudaMemsetAsync(w->AQ, 0, nP * sizeof(float), st));
  if (ne) {
    CK(cudaMemsetAsync(w->AL, 0, ne * sizeof(float), st));
    CK(cudaMemsetAsync(w->APp, 0, 2 * ne * sizeof(float), st));
  }
  const AdjArgs r = adj_args(h);
  int rc;
  if (w->g_N != w->N || w->g_m != w->m || w->g_mask != r.mask) {
    adj_drop_graphs(w);
    w->graphs.assign(w->nck, nullptr);
    w->g_N = w->N;
    w->g_m = w->m;
    w->g_mask = r.mask;
  }
  for (int c = w->nck - 1; c >= 0; --c) {
    if (h->prof) {  // measurement hooks need direct launches
      if ((rc = adj_segment(h, r, c))) return rc;
      continue;
    }
    if (!w->graphs[c] && (rc = adj_capture_segment(h, r, c, &w->graphs[c]))) return rc;
    CK(cudaGraphLaunch(w->graphs[c], st));
  }
  CK(launch_adj_initial(r, st));
  CK(launch_sum_f64(w->Aal, nal, h->partials, h->counter, h->red_out, st));
  CK(cudaMemcpyAsync(grad_f_dev, w->Af, h->npx * sizeof(float), cudaMemcpyDeviceToDevice, st));
  double ga = 0.0;
  CK(cudaMemcpyAsync(&ga, h->red_out, sizeof(double), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  if ((rc = check_timeout(h))) return rc;
  *grad_alpha = ga;
  return DD_TV_OK;
}

int dd_tv_adjoint_release(dd_tv* h) {
  if (!h) return DD_TV_EINVAL;
  if (h->adj) {
    CK(cudaStreamSynchronize(h->stream));
    adj_free(h->adj);
    h->adj = nullptr;
  }
  return DD_TV_OK;
}

int dd_tv_profile_read(dd_tv* h, double* ms, long long* launches) {
  if (!h) return DD_TV_EINVAL;
  CK(cudaStreamSynchronize(h->stream));
  int rc = check_timeout(h);
  if (rc) return rc;
  double acc[3] = {0.0, 0.0, 0.0};
  for (auto& m : h->marks) {
    float t = 0.f;
    if (cudaEventElapsedTime(&t, m.a, m.b) == cudaSuccess) acc[m.slot] += t;
    cudaEventDestroy(m.a);
    cudaEventDestroy(m.b);
  }
  h->marks.clear();
  for (int s = 0; s < 3; ++s) {
    if (ms) ms[s] = acc[s];
    if (launches) launches[s] = h->prof_launches[s];
    h->prof_launches[s] = 0;
  }
  return DD_TV_OK;
}

int dd_tv_fault_probe(dd_tv* h, int kind, double* waited_ms) {
  if (!h) return DD_TV_EINVAL;
  if (waited_ms) *waited_ms = 0.0;
  if (kind == 0) {
    unsigned long long* d_ns = nullptr;
    CK(cudaMalloc((void**)&d_ns, sizeof(*d_ns)));
    unsigned long long ns = 0;
    cudaError_t e = launch_wait_probe(h->flag, d_ns, h->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&ns, d_ns, sizeof(ns), cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    cudaFree(d_ns);
    if (e != cudaSuccess) return fail(h, DD_TV_ECUDA, "wait probe: %s", cudaGetErrorString(e));
    if (waited_ms) *waited_ms = (double)ns * 1e-6;
  } else if (kind == 1) {
    const int one = 1;
    CK(cudaMemcpyAsync(h->flag, &one, sizeof(int), cudaMemcpyHostToDevice, h->stream));
  } else {
    return fail(h, DD_TV_EINVAL, "fault probe kind must be 0 (device wait) or 1 (status word)");
  }
  return check_timeout(h);
}

}  // extern "C"

// ---- row-block shards (dd_tv_create_shard)

int dd_tv_shard_rows(const dd_tv* h, int* row_begin, int* rows) {
  if (!h) return DD_TV_EINVAL;
  if (row_begin) *row_begin = h->shard ? h->row0 : 0;
  if (rows) *rows = h->g.H;
  return DD_TV_OK;
}

int dd_tv_shard_export(dd_tv* h, float* top_dev, float* bottom_dev) {
  if (!h) return DD_TV_EINVAL;
  if (!h->shard) return fail(h, DD_TV_EINVAL, "not a shard");
  const Grid& g = h->g;
  if ((g.cut_top && !top_dev) || (g.cut_bot && !bottom_dev))
    return fail(h, DD_TV_EINVAL, "a buffer is required for every cut side (top %d, bottom %d)", g.cut_top, g.cut_bot);
  // this shard's copies on its cut sides of p~^n, n = outer iterations run: the t-side
  // copy of the line above (its top side) and the s-side copy of the line below
  const Strips& s = h->strips[h->n & 1];
  const size_t W = (size_t)g.W;
  if (g.cut_top) CK(cudaMemcpyAsync(top_dev, s.ST, W * sizeof(float), cudaMemcpyDeviceToDevice, h->stream));
  if (g.cut_bot)
    CK(cudaMemcpyAsync(bottom_dev, s.SB + (h->nlh - 1) * W, W * sizeof(float), cudaMemcpyDeviceToDevice, h->stream));
  return DD_TV_OK;
}

int dd_tv_shard_import(dd_tv* h, const float* above_dev, const float* below_dev) {
  if (!h) return DD_TV_EINVAL;
  if (!h->shard) return fail(h, DD_TV_EINVAL, "not a shard");
  const Grid& g = h->g;
  if ((g.cut_top && !above_dev) || (g.cut_bot && !below_dev))
    return fail(h, DD_TV_EINVAL, "a buffer is required for every cut side (top %d, bottom %d)", g.cut_top, g.cut_bot);
  // the neighbours' copies of the same p~^n: the s-side copy of the line above (the
  // bottom side of the shard above) and the t-side copy of the line below
  const Strips& s = h->strips[h->n & 1];
  const size_t W = (size_t)g.W;
  if (g.cut_top) CK(cudaMemcpyAsync(s.SB, above_dev, W * sizeof(float), cudaMemcpyDeviceToDevice, h->stream));
  if (g.cut_bot)
    CK(cudaMemcpyAsync(s.ST + (h->nlh - 1) * W, below_dev, W * sizeof(float), cudaMemcpyDeviceToDevice, h->stream));
  return DD_TV_OK;
}

int dd_tv_shard_edge_rows(dd_tv* h, float* first_row_dev, float* last_row_dev) {
  if (!h) return DD_TV_EINVAL;
  if (!h->loaded) return fail(h, DD_TV_EINVAL, "no data loaded");
  const size_t W = (size_t)h->g.W;
  if (first_row_dev) CK(cudaMemcpyAsync(first_row_dev, h->u, W * sizeof(float), cudaMemcpyDeviceToDevice, h->stream));
  if (last_row_dev)
    CK(cudaMemcpyAsync(last_row_dev, h->u + (size_t)(h->g.H - 1) * W, W * sizeof(float), cudaMemcpyDeviceToDevice,
                       h->stream));
  return DD_TV_OK;
}

int dd_tv_shard_energy(dd_tv* h, const float* row_below_dev, double* J_out) {
  if (!h) return DD_TV_EINVAL;
  if (!h->loaded) return fail(h, DD_TV_EINVAL, "no data loaded");
  if (!J_out) return fail(h, DD_TV_EINVAL, "J_out is NULL");
  if (h->g.cut_bot && !row_below_dev) return fail(h, DD_TV_EINVAL, "the bottom side is cut: row_below is required");
  double o[2];
  int rc = energy_of(h, h->u, h->f, h->has_mask ? h->mask : nullptr, false, o);
  if (rc) return rc;
  double cut = 0.0;
  if (h->g.cut_bot) {
    CK(launch_row_tv(row_below_dev, h->u + (size_t)(h->g.H - 1) * h->g.W, h->g.W, h->red_out + 1, h->stream));
    CK(cudaMemcpyAsync(&cut, h->red_out + 1, sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
  }
  *J_out = o[0] + cut;
  return DD_TV_OK;
}
