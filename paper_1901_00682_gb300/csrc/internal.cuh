// Internal declarations shared by the translation units of the dd_tv library.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "pointwise.cuh"

namespace ddtv {

// Image and subdomain grid.  cut_top / cut_bot: the top side of tile row 0 / the
// bottom side of tile row NR-1 lies on an interface with a neighbouring row-block
// shard (its dofs are active, its multipliers and strips sit one line before / after
// the handle's own lines); 0 for a whole image, where those sides are on the image
// boundary.
struct Grid {
  int H, W, NR, NC;
  int cut_top = 0, cut_bot = 0;
};

// Interface strips: the interface values of one torn dual field p~^n.
//   SB (NR-1) x W : bottom side of tile row a (s-side copy of horizontal interface a)
//   ST (NR-1) x W : top side of tile row a+1  (t-side copy)
//   SR (NC-1) x H : right side of tile column b (s-side copy of vertical interface b)
//   SL (NC-1) x H : left side of tile column b+1 (t-side copy)
struct Strips {
  float *SB, *ST, *SR, *SL;
};

// Arguments of one local-solve launch (fused or plain path).
struct LocalArgs {
  Grid g;
  int K;                 // inner iterations
  float tau;             // outer tau (proximal centre phat = p~ -+ tau lambda)
  float c1, c2;          // SEG constants
  const float* f;        // H x W
  const uint8_t* mask;   // H x W or nullptr
  float* u;              // H x W
  float* P1;             // (H + NR) x W torn
  float* P2;             // H x (W + NC) torn
  const float* lamh;     // (NR-1) x W
  const float* lamv;     // (NC-1) x H
  Strips out;            // strips of p~^{n+1} (written at the end)
  const Coef* coef;      // K coefficient sets (device)
  int* err;              // set non-zero by a kernel whose bounded wait ran out
  // adaptive inner stopping (eq. stop_inner1); inner_tol2 = 0 selects K fixed iterations
  double inner_tol2;               // tol^2: stop once sum (dp)^2 < tol^2 sum p^2
  int* inner_used;                 // NR * NC: inner iterations of each tile, last launch
  int* inner_max;                  // running maximum of inner_used
  unsigned long long* inner_work;  // running sum of tile pixels x inner iterations
};

// Batch of images solved together (every image partitioned into exact 128 x 128
// subdomains).  Device arrays, one entry per image unless stated otherwise.
struct BatchArgs {
  const LocalArgs* args;   // per-image descriptor (its `out` field is unused)
  const Strips* strips;    // 2 per image: strip sets by parity
  const int* fid;          // fidelity per image
  const int* tile_img;     // per tile of the batch: its image
  const int* tile_base;    // first batch tile of each image
  int write_set;           // strip set receiving p~^{n+1}
};

// Batched multiplier update: per image interface elements in units of 4 edges.
struct BatchIfaceArgs {
  const LocalArgs* args;   // per-image descriptor (geometry, lamh, lamv)
  const Strips* strips;    // 2 per image
  const float* sigma;      // outer sigma per image
  const int* elem_base;    // n_img + 1 prefix sums of (nh + nv) / 4
  int n_img;
  int cur_set;             // strip set holding p~^n
};

// Adjoint fields of the reverse pass (kernels_adjoint.cu).  A* is the adjoint of the
// named forward quantity; AP/AQ/APh live on the torn layout of P1/P2.
struct AdjArgs {
  Grid g;
  int fid;
  float c1, c2;
  const float* f;          // H x W
  const uint8_t* mask;     // H x W or nullptr
  float *Au, *Ad, *Af;     // H x W: u, div pbar (scaled), f
  double* Aal;             // adj_alpha_slots(g) per-block partial sums of the alpha adjoint
  const int4* rowtab;      // H: (tile row, first row, end row) of every pixel row
  const int4* coltab;      // W: (tile column, first column, end column) of every pixel column
  float *AP1, *AP2;        // p
  float *AQ1, *AQ2;        // pbar
  float *APh1, *APh2;      // phat
  float *ALh, *ALv;        // lambda
  Strips APp;              // interface values of p~^{n-1}
  float* tape;             // tile-fused reverse kernel: adj_fused_tape_floats(g, K) floats
};

// ---- kernels_interface.cu
// lambda += sigma ((2 cur_s - prev_s) - (2 cur_t - prev_t)) on every interface edge.
cudaError_t launch_interface(const Grid& g, float sigma, Strips cur, Strips prev, float* lamh, float* lamv,
                             cudaStream_t st);
// strips <- interface values of the torn field (P1, P2)
cudaError_t launch_extract_strips(const Grid& g, const float* P1, const float* P2, Strips s, cudaStream_t st);
// P1/P2 <- 0 except the interface values, taken from the strips
cudaError_t launch_scatter_strips(const Grid& g, Strips s, float* P1, float* P2, cudaStream_t st);

cudaError_t launch_interface_batch(const BatchIfaceArgs& a, int total4, cudaStream_t st);

// ---- kernels_fused.cu
// All tiles of all images of a batch, one launch (BatchArgs.write_set selects the strips);
// tile: the subdomain side, 128 (persistent micro-tile kernels: variant 0 the 4 x 4 one
// when K <= fused_mt4_max_inner(), else and for variant 2 the 2 x 4 one) or 64 (one CTA
// per subdomain).
cudaError_t launch_fused_batch(const BatchArgs& B, int total_tiles, int tile, int variant, int K, cudaStream_t st);
// One outer iteration's local solves, all tiles, fused (returns cudaErrorInvalidValue
// if no fused configuration fits the tile shape).
cudaError_t launch_fused_local(const LocalArgs& a, int fidelity, int variant, cudaStream_t st);
// Sets the shared-memory opt-in of every fused configuration on the current device
// (called at handle creation, outside any stream capture).
cudaError_t fused_prepare();
// Largest tile (rows, cols) the fused kernel supports.
void fused_max_tile(int* rows, int* cols);
// Number of hardware mappings available for 128 x 128 tiles.
int fused_num_variants();
// Name of the configuration chosen for a tile shape and variant (for reports).
const char* fused_config_name(int mr, int mc, int variant);

// ---- kernels_fused_mt.cu
// Persistent fused local solver on 2 x 4 micro-tiles (two columns by four rows per
// thread); 128 x 128 tiles with u, f, P1 16-byte aligned (fused_mt_supported).
bool fused_mt_supported(const LocalArgs& a);
cudaError_t launch_fused_mt(const LocalArgs& a, int fidelity, cudaStream_t st);
cudaError_t fused_mt_prepare();
// The same kernel over the work list of a batch (every image's arrays 16-byte aligned).
cudaError_t launch_fused_mt_batch(const BatchArgs& B, int total_tiles, cudaStream_t st);

// ---- kernels_fused_mt4.cu
// Persistent fused local solver on 4 x 4 micro-tiles, one warp per thread row, three
// 128-thread CTAs per SM; 128 x 128 tiles with 16-byte aligned rows
// (fused_mt4_supported).
bool fused_mt4_supported(const LocalArgs& a);
// tma: move the state with tensor copies (falls back to cp.async if the tensor maps
// cannot be encoded).  With a.inner_tol2 > 0 (adaptive inner stop) the tensor-copy
// kernel runs whatever tma says, and cudaErrorNotSupported comes back if its maps
// cannot be encoded.
cudaError_t launch_fused_mt4(const LocalArgs& a, int fidelity, bool tma, cudaStream_t st);
cudaError_t fused_mt4_prepare();
// The same kernel (cp.async copies) over the work list of a batch: every image's arrays
// 16-byte aligned, inner count <= fused_mt4_max_inner().
cudaError_t launch_fused_mt4_batch(const BatchArgs& B, int total_tiles, cudaStream_t st);
int fused_mt4_max_inner();

// ---- kernels_plain.cu
// phat = p~ -+ tau lambda on the interface sides, pbar = p~; full arrays.
cudaError_t launch_plain_phat(const LocalArgs& a, float* Ph1, float* Ph2, float* Pb1, float* Pb2, cudaStream_t st);
// one u-step over the whole torn field (reads pbar)
cudaError_t launch_plain_ustep(const LocalArgs& a, const float* Pb1, const float* Pb2, const Coef* ck, int fidelity,
                               cudaStream_t st);
// one p-step; phat may be nullptr (no proximal term, full-dimension comparator);
// write_strips: also write the interface strips of the new p.
cudaError_t launch_plain_pstep(const LocalArgs& a, const float* Ph1, const float* Ph2, float* Pb1, float* Pb2,
                               const Coef* ck, bool write_strips, cudaStream_t st);

// ---- kernels_reduce.cu
// out[0] = J(u) = alpha F(u) + TV(u); out[1] = dual value of the averaged torn field
// (P1, P2 nullable: then out[1] is not computed).  partials: scratch of
// reduce_partials_count() doubles; counter: one zeroed unsigned int that the kernel
// leaves zeroed.
cudaError_t launch_energy(const Grid& g, int fidelity, float alpha, float c1, float c2, const float* u,
                          const float* f, const uint8_t* mask, const float* P1, const float* P2, double* partials,
                          unsigned int* counter, double* out, cudaStream_t st);
int reduce_partials_count();
// out[0] = sum_j |a_j - b_j|, j < n (float64, deterministic)
cudaError_t launch_row_tv(const float* a, const float* b, int n, double* out, cudaStream_t st);

// ---- kernels_adjoint.cu
// u-step / p-step of the plain path that also record ubar (H x W) and the projection's
// pass bit of every active dof (M1 (H+NR) x W, M2 H x (W+NC); inactive dofs untouched).
// rt / ct: the row and column tables of AdjArgs.
cudaError_t launch_ustep_tape(const LocalArgs& a, const int4* rt, const int4* ct, const float* Pb1, const float* Pb2,
                              const Coef* ck, int fidelity, float* ubar_out, cudaStream_t st);
cudaError_t launch_pstep_tape(const LocalArgs& a, const int4* rt, const int4* ct, const float* Ph1, const float* Ph2,
                              float* Pb1, float* Pb2, const Coef* ck, uint8_t* M1, uint8_t* M2, cudaStream_t st);
// reverse of one inner iteration (two kernels); first / last as in adj_dof
cudaError_t launch_adj_inner(const AdjArgs& r, const Coef* ck, const float* ubar, const uint8_t* M1,
                             const uint8_t* M2, bool first, bool last, cudaStream_t st);
// reverse of the multiplier update and proximal centre of one outer iteration
cudaError_t launch_adj_interface(const AdjArgs& r, float sigma, float tau, cudaStream_t st);
// Af += du^0/df Au
cudaError_t launch_adj_initial(const AdjArgs& r, cudaStream_t st);
// out[0] = sum of x[0..n) (partials: sum_f64_partials_count() doubles; counter zeroed)
cudaError_t launch_sum_f64(const double* x, long long n, double* partials, unsigned int* counter, double* out,
                           cudaStream_t st);
int sum_f64_partials_count();
// number of float64 partial sums the reverse u-kernel keeps for an image grid
long long adj_alpha_slots(const Grid& g);

// ---- kernels_adjoint_fused.cu
// Reverse of one outer iteration's local solves, tape in shared memory: a = the local
// solve's arguments (state after the multiplier update), z = the adjoint fields (Au,
// AP1/AP2 in: adjoints of u^{n+1}, p~^{n+1}; out: of u^n and of p~^n through the local
// solve; APh1/APh2 out on the subdomain sides; Af +=; Aal += per (tile, CTA) slot).
cudaError_t launch_adj_fused(const LocalArgs& a, const AdjArgs& z, int fidelity, cudaStream_t st);
// floats of the fused reverse kernel's tape (0 if the tile shape is not supported)
size_t adj_fused_tape_floats(const Grid& g, int K);
// shared-memory opt-in of the fused reverse kernels (outside any stream capture)
cudaError_t adj_fused_prepare();
// alpha partial-sum slots the fused reverse kernel uses
long long adj_alpha_slots_fused(const Grid& g);

// ---- kernels_misc.cu
// u0 = f (0 on D) for L2/L1, 1/2 for SEG
cudaError_t launch_init_u(const Grid& g, int fidelity, const float* f, const uint8_t* mask, float* u, cudaStream_t st);
// one bounded mbarrier wait that runs out (nothing completes the phase): sets *err,
// writes the device time it took (ns) to *waited_ns
cudaError_t launch_wait_probe(int* err, unsigned long long* waited_ns, cudaStream_t st);
// global field (H+1) x W / H x (W+1) <-> torn field with a 1 x 1 grid (same arrays)
}  // namespace ddtv
