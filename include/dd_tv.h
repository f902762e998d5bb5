/*
 * dd_tv.h - C ABI of the GB300 (sm_103a) solver for the primal-dual domain
 * decomposition method for dual total variation minimisation of Lee & Park,
 * "A finite element nonoverlapping domain decomposition method with Lagrange
 * multipliers for the dual total variation minimizations" (Algorithm 1).
 *
 * Problem (Section 3, eq. model):  min_u  J(u) = alpha F(u) + TV(u)  on an H x W
 * image of unit square pixels, TV the anisotropic discrete total variation (the
 * proposition on the FE/FD equivalence), with one of the fidelities of Section 3:
 *   DD_TV_L2  : F = 1/2 sum_{T not in D} (u - f)^2     ROF denoising / L2 inpainting
 *   DD_TV_L1  : F =     sum_{T not in D} |u - f|       TV-L1 denoising / L1 inpainting
 *   DD_TV_SEG : F = <u, g> + chi_{[0,1]}(u),  g = (f - c1)^2 - (f - c2)^2
 *                                                      convex Chan-Vese segmentation
 * D is the optional inpainting domain (mask byte 1 = pixel in D, f ignored there).
 *
 * Method (Algorithm 1): the image is split into sub_rows x sub_cols rectangles
 * (Section 2.4); tile row a covers pixel rows [floor(a H / sub_rows),
 * floor((a+1) H / sub_rows)), tile columns likewise.  Each outer iteration
 *   lambda <- lambda + sigma B (2 p~^n - p~^{n-1})         (interface multipliers)
 *   phat   <- p~^n - tau B^* lambda                         (proximal centre)
 *   every tile, in parallel: inner_iters accelerated primal-dual iterations on its
 *   local saddle problem (Section 5, eq. local), warm-started from (u^n, p~^n).
 * p~ is the torn lowest-order Raviart-Thomas dual field: one normal component per
 * pixel edge, every tile keeping its own copy on its sides (Section 2.4).
 *
 * Conventions for every entry point:
 *   - images are row-major float32 H x W (u, f) or uint8 H x W (mask);
 *   - "_host" pointers are ordinary host memory, "_dev" pointers device memory of
 *     the current CUDA device; the library never keeps a caller's pointer after
 *     the call returns, and the caller keeps ownership of everything it passes;
 *   - calls return a dd_tv_status; on failure dd_tv_last_error(h) describes it;
 *     no call aborts the process or traps the GPU;
 *   - work is issued on the handle's stream (dd_tv_set_stream); calls that return
 *     a host value or write host memory synchronise that stream first.
 * The handle owns all device memory it uses; it is not thread-safe.
 */
#ifndef DD_TV_H
#define DD_TV_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct dd_tv dd_tv;

typedef enum { DD_TV_L2 = 0, DD_TV_L1 = 1, DD_TV_SEG = 2 } dd_tv_fidelity;

typedef enum {
  DD_TV_OK = 0,
  DD_TV_EINVAL = 1,      /* invalid argument (message in dd_tv_last_error)            */
  DD_TV_ENOMEM = 2,      /* device or host allocation failed                           */
  DD_TV_ECUDA = 3,       /* a CUDA call failed                                         */
  DD_TV_ETIMEOUT = 4,    /* a bounded device-side wait ran out                          */
  DD_TV_ENOTCONV = 5,    /* outer_tol given and not reached within outer_iters          */
  DD_TV_EUNSUPPORTED = 6 /* valid problem outside what the chosen path implements       */
} dd_tv_status;

/* Which implementation runs an outer iteration. */
typedef enum {
  DD_TV_PATH_FUSED = 0,  /* interface kernel + fused subdomain-per-cluster local solver */
  DD_TV_PATH_PLAIN = 1,  /* one global-memory kernel per step (comparator)              */
  DD_TV_PATH_FULLDIM = 2 /* undecomposed primal-dual iteration, N = 1 (Section 5 "CP")  */
} dd_tv_path;

typedef struct {
  int height, width;      /* H, W > 0                                                      */
  int sub_rows, sub_cols; /* 1 <= sub_rows <= H, 1 <= sub_cols <= W (Section 2.4)          */
  int fidelity;           /* dd_tv_fidelity                                                */
  double alpha;           /* > 0 (eq. model)                                               */
  double c1, c2;          /* DD_TV_SEG region constants (eq. CCV)                           */
  int outer_iters;        /* >= 0: outer iterations run by dd_tv_solve*                      */
  int inner_iters;        /* 1..DD_TV_MAX_INNER: local iterations per outer iteration         */
  double tau, sigma;      /* outer steps, tau sigma <= 1/2 (Algorithm 1; Section 5 uses
                             tau = 50, sigma tau = 1/2; tau = 1 for segmentation)           */
  double tau0, sigma0;    /* initial local steps on p and u (Section 5: 10 and 1/80)         */
  double gamma;           /* local acceleration, 0 < gamma <= 1/tau (Section 5: 1/(8 tau))   */
  double outer_tol;       /* > 0: stop once (J(u^n) - energy_ref)/|energy_ref| <= outer_tol  */
  double energy_ref;      /* J* used by outer_tol (eq. stop_outer)                           */
  int energy_every;       /* with outer_tol: evaluate J every energy_every outer iterations  */
  int path;               /* dd_tv_path                                                    */
  int variant;            /* fused path, hardware mapping of exact 128 x 128 subdomains:
                             0 persistent 4 x 4 micro-tiles, state moved by tensor
                             copies (default); 1 the same with cp.async copies; 2
                             persistent 2 x 4 micro-tiles; 3 one cluster per subdomain
                             with cluster barriers (the kernel of every other tile
                             shape).  The arithmetic and results do not depend on it  */
  double inner_tol;       /* >= 0.  0: every local solve runs inner_iters iterations.  > 0:
                             adaptive inner stopping (Section 5, eq. stop_inner1): a
                             subdomain stops after the first inner iteration k with
                             ||p^{k+1} - p^k||_2 < inner_tol ||p^{k+1}||_2 (norms over its
                             dual dofs; p^{k+1} = 0 counts as converged), at most
                             inner_iters iterations.  The decision is taken in float64 on
                             float32 sums of squares.  Fused path only (the other paths
                             return DD_TV_EUNSUPPORTED); the fused kernel then runs a
                             cluster-wide reduction every inner iteration.           */
} dd_tv_params;

#define DD_TV_MAX_INNER 1024

typedef struct {
  int outer_done;         /* outer iterations run by the call                              */
  long long pixel_iters;  /* inner work units: sum over outer iterations and subdomains of
                             (subdomain pixels x inner iterations run); H * W * inner_iters
                             * outer_done without inner_tol                              */
  double energy;          /* J(u) at exit; NaN when not evaluated                          */
  double rel_err;         /* (energy - energy_ref)/|energy_ref|; NaN when not evaluated     */
  double ms;              /* device time of the outer iterations (CUDA events)             */
  int converged;          /* 1 if outer_tol was reached                                    */
  int inner_max;          /* most inner iterations any subdomain ran in one outer iteration
                             of the call (the paper's "max inner iter"; = inner_iters
                             without inner_tol)                                          */
} dd_tv_stats;

/* Fills p with the paper's experimental settings (Section 5): tau = 50,
 * sigma = 1/(2 tau), tau0 = 10, sigma0 = 1/80, gamma = 1/(8 tau), inner_iters = 10,
 * fidelity L2, alpha = 10, one subdomain, the fused path, no outer_tol. */
void dd_tv_default_params(dd_tv_params* p);

/* Validates p and allocates the device state for one H x W problem.  *out is set to
 * a new handle (or NULL on error).  Must be called with the target device current. */
int dd_tv_create(dd_tv** out, const dd_tv_params* p);

/* Frees the handle and its device memory.  NULL-safe. */
int dd_tv_destroy(dd_tv* h);

/* Human-readable description of the last error on h (static string for h == NULL). */
const char* dd_tv_last_error(const dd_tv* h);

/* Sets the stream (a cudaStream_t, 0 = legacy default) all later work is issued on. */
int dd_tv_set_stream(dd_tv* h, void* stream);

/* Full solve from host memory: copies f_host (and mask_host, nullable) to the device,
 * initialises the state (u^0 = f with f := 0 on D, or 1/2 for DD_TV_SEG; p~ = 0,
 * lambda = 0), runs outer_iters outer iterations (or until outer_tol), copies u to
 * u_host.  stats is nullable.  Synchronous. */
int dd_tv_solve(dd_tv* h, const float* f_host, const uint8_t* mask_host, float* u_host, dd_tv_stats* stats);

/* The same with device buffers; asynchronous on the handle's stream unless
 * stats != NULL or outer_tol > 0 (both need host-side values). */
int dd_tv_solve_device(dd_tv* h, const float* f_dev, const uint8_t* mask_dev, float* u_dev, dd_tv_stats* stats);

/* Stepping interface.  dd_tv_load copies f (and mask) from device memory into the
 * handle and initialises the state as dd_tv_solve does; dd_tv_iterate runs n_outer
 * outer iterations on the resident state (asynchronous); dd_tv_get_u copies the
 * current u to u_dev. */
int dd_tv_load(dd_tv* h, const float* f_dev, const uint8_t* mask_dev);
int dd_tv_iterate(dd_tv* h, int n_outer);
int dd_tv_get_u(dd_tv* h, float* u_dev);

/* Inner iterations run by every subdomain (row-major subdomain order, sub_rows x
 * sub_cols ints, host memory) in the last outer iteration, and the largest count of
 * any subdomain in any outer iteration since the last load, solve or call of this
 * function (*max_out, nullable; the counter is then reset).  Without inner_tol
 * every count is inner_iters (0 before the first outer iteration).  Synchronous. */
int dd_tv_inner_counts(dd_tv* h, int* counts_host, int* max_out);

/* Number of outer iterations run since the last dd_tv_load / dd_tv_set_state. */
int dd_tv_outer_count(const dd_tv* h);

/* State exchange in the torn layout (device buffers, float32, caller-allocated):
 *   u     H x W
 *   P1    (H + sub_rows) x W      tile row a owns rows r0(a)+a .. r0(a+1)+a: the
 *                                 normal components (oriented down) on the horizontal
 *                                 edges of that tile row, its top and bottom sides
 *                                 included (0 on the image boundary)
 *   P2    H x (W + sub_cols)      tile column b owns columns c0(b)+b .. c0(b+1)+b
 *                                 (normal components oriented right)
 *   lamh  (sub_rows - 1) x W      multiplier of the edge between tile rows a, a+1
 *   lamv  (sub_cols - 1) x H      multiplier of the edge between tile columns b, b+1
 *   P1prev, P2prev                p~^{n-1} in the P1/P2 layout (only its interface
 *                                 values are used; get writes zeros elsewhere)
 * Pointers for empty arrays (e.g. lamh with sub_rows = 1) may be NULL.  For the
 * full-dimension path P1/P2 hold the global field (sub grid 1 x 1) and P1prev/P2prev
 * the extrapolated field pbar. */
int dd_tv_get_state(dd_tv* h, float* u, float* P1, float* P2, float* lamh, float* lamv, float* P1prev,
                    float* P2prev);
int dd_tv_set_state(dd_tv* h, const float* u, const float* P1, const float* P2, const float* lamh,
                    const float* lamv, const float* P1prev, const float* P2prev, int outer_count);

/* J(u) = alpha F(u) + TV(u) (eq. model) of a device image u_dev against the data
 * f_dev / mask_dev (mask nullable) with the handle's fidelity, alpha, c1, c2.  Kahan-
 * compensated float32 per thread, float64 across threads and blocks, fixed order
 * (deterministic).  Synchronous; writes *J_out. */
int dd_tv_energy(dd_tv* h, const float* u_dev, const float* f_dev, const uint8_t* mask_dev, double* J_out);

/* Energy of the current iterate and the dual value of the averaged dual field
 * (duality-gap certificate: d <= J* <= J): L2 without mask:
 * -(1/(2 alpha)) ||div p + alpha f||^2 + (alpha/2) ||f||^2; SEG: sum min(0, alpha g -
 * div p); otherwise *D_out = -inf.  Synchronous. */
int dd_tv_gap(dd_tv* h, double* J_out, double* D_out);


/* Energy J(u) of the current iterate (the quantity of the outer stopping rule,
 * eq. stop_outer).  Synchronous. */
int dd_tv_current_energy(dd_tv* h, double* J_out);

/* ---- Measurement hooks (no counterpart in the paper). ----
 * dd_tv_set_profiling(h, 1): later dd_tv_iterate / energy calls launch their kernels
 * directly (no graph replay) and bracket every phase with CUDA events on the
 * handle's stream.  dd_tv_profile_read synchronises and writes, for each phase
 * (0 = interface multiplier update, 1 = local solves, 2 = energy reduction), the
 * summed device time in milliseconds and the number of kernel launches since
 * profiling was switched on (arrays of 3; either pointer may be NULL); it then
 * resets the counters.  dd_tv_set_profiling(h, 0) returns to graph replay. */
int dd_tv_set_profiling(dd_tv* h, int on);
int dd_tv_profile_read(dd_tv* h, double* ms, long long* launches);

/* ---- Failure-detection hook (no counterpart in the paper). ----
 * Every wait of the fused kernels on a halo or a copy (an mbarrier phase) is bounded
 * (a thousand suspended mbarrier.try_wait rounds: 3.8 ms measured on GB300); when the
 * bound runs out the kernel sets the handle's device status word and goes on, so a
 * launch whose waits all run out still ends (within about 2 s at the 4096^2 size),
 * and the next call that synchronises returns DD_TV_ETIMEOUT.
 * dd_tv_fault_probe makes that happen on purpose without a fault: kind 0 launches one
 * thread that waits, with the same bounded wait, on an mbarrier phase that nothing
 * completes (no copy is counted on it); kind 1 writes the status word from the host,
 * as a corrupted word would read.  Either way the call then reads the word as the
 * solver does and returns DD_TV_ETIMEOUT (message in dd_tv_last_error), the word is
 * cleared and the handle stays usable.  *waited_ms (may be NULL) receives the device
 * time the kind-0 wait took (0 for kind 1).  Other kinds: DD_TV_EINVAL. */
int dd_tv_fault_probe(dd_tv* h, int kind, double* waited_ms);

/* Measures the shared-memory load bandwidth of the current device (bytes per second
 * summed over all SMs) with a streaming ld.shared loop, for use as the roofline
 * denominator of the fused local solver.  Synchronous; allocates and frees its own
 * small device buffer.  *gbs_out is in GB/s (1e9 bytes/s). */
int dd_tv_measure_smem_bandwidth(double* gbs_out);

/* Energy J(u) = alpha F(u) + TV(u), like dd_tv_energy, for callers that cannot
 * allocate device memory at the time they need it (for instance a process whose
 * device memory is entirely held by another framework's pool, or a latency-critical
 * loop that must not pay cudaMalloc's implicit synchronisation).  The paper has no
 * counterpart: this is a deployment variant of the energy reduction.
 *
 * No handle and no allocation: the reduction's scratch is a fixed 9,760-byte array
 * in the library's device memory (every GPU that loads the library holds it until
 * the process exits).  The first call on a device looks that array's address up with
 * the device current, so make the first call on each device outside any stream
 * capture.  Images of up to 2^31 - 1 pixels are accepted; larger ones, a null
 * pointer, a bad fidelity or alpha <= 0 return DD_TV_EINVAL.  u_dev, f_dev, mask_dev
 * (nullable) are H x W device images as in dd_tv_energy; the caller keeps them.
 * stream is a cudaStream_t (0 = legacy default stream).  All calls share the one
 * scratch array, so calls whose work overlaps on the GPU (other streams or threads)
 * race and may return wrong values; serialise them.  Synchronous: waits for the
 * stream and writes *J_out. */
int dd_tv_energy_noalloc(const float* u_dev, const float* f_dev, const uint8_t* mask_dev, int height, int width,
                         int fidelity, double alpha, double c1, double c2, void* stream, double* J_out);

/* ---- Row-block shards: one problem over several GPUs (one process per GPU).
 * Algorithm 1 couples the subdomains only through the multiplier update on the
 * interfaces (its first line: lambda^{n+1} = lambda^n + sigma B (2 p~^n - p~^{n-1})),
 * so a contiguous block of tile rows can live on each GPU.  A shard handle owns tile
 * rows [tile_row_begin, tile_row_end) of the problem p describes (the whole image's
 * height, width and subdomain grid): its image is rows [row_begin, row_begin + rows)
 * of f (dd_tv_shard_rows), which dd_tv_load takes as an ordinary rows x width device
 * image.  The sides of its first and last tile rows that face another shard are
 * interface sides ("cut"): their dual dofs are active, and the shard keeps its own
 * copy of the multipliers on the cut lines.  Both shards beside a cut update those
 * multipliers from the same four strips with the same float32 arithmetic, so the copies
 * stay equal bit for bit; the only data that crosses is, per outer iteration, each
 * shard's copy of p~^n on its cut sides (width floats per cut), and for the energy its
 * first pixel row.  A run of S shards reproduces the single-handle run bit for bit.
 *
 * Per outer iteration: dd_tv_iterate(h, 1); dd_tv_shard_export into two width-float
 * device buffers; send the top buffer to the shard above and the bottom one to the
 * shard below (NCCL, or copies), receive theirs; dd_tv_shard_import.  The first outer
 * iteration needs no exchange (p~^0 = p~^{-1} = 0).
 *
 * Requirements: the fused path, a fixed inner iteration count (inner_tol = 0), tile
 * rows of equal height (height a multiple of sub_rows).  Errors: DD_TV_EINVAL for a
 * bad range or uneven tile rows, DD_TV_EUNSUPPORTED for another path or inner_tol > 0.
 * On a shard, dd_tv_iterate accepts one outer iteration per call, and dd_tv_solve,
 * dd_tv_solve_device, dd_tv_get_state, dd_tv_set_state, dd_tv_gap and the adjoint
 * calls return DD_TV_EUNSUPPORTED. */
int dd_tv_create_shard(dd_tv** out, const dd_tv_params* p, int tile_row_begin, int tile_row_end);
/* First image row and number of rows of the handle's image (0 and height for a whole
 * image). */
int dd_tv_shard_rows(const dd_tv* h, int* row_begin, int* rows);
/* Copies the shard's own copies of p~^n (n = outer iterations run) on its cut sides:
 * top_dev <- the normal components on its top side (width floats), bottom_dev <- those
 * on its bottom side.  A buffer is required for each cut side and ignored otherwise.
 * Asynchronous on the handle's stream. */
int dd_tv_shard_export(dd_tv* h, float* top_dev, float* bottom_dev);
/* Takes the neighbours' copies of p~^n on the same lines: above_dev from the shard
 * above (its bottom side), below_dev from the shard below (its top side).  Call after
 * dd_tv_iterate and before the next one.  Asynchronous on the handle's stream. */
int dd_tv_shard_import(dd_tv* h, const float* above_dev, const float* below_dev);
/* Copies the first and the last pixel row of the current u (width floats each; either
 * pointer may be NULL).  Asynchronous. */
int dd_tv_shard_edge_rows(dd_tv* h, float* first_row_dev, float* last_row_dev);
/* The shard's part of J(u) = alpha F(u) + TV(u) (eq. model): alpha F and TV over its
 * rows plus sum_j |u_below(0, j) - u(rows - 1, j)| across its bottom cut, row_below_dev
 * being the first row of the shard below (required when the bottom side is cut).  The
 * parts of all shards add up to J of the whole image.  Synchronous. */
int dd_tv_shard_energy(dd_tv* h, const float* row_below_dev, double* J_out);

/* ---- Batched solve (many images in one launch per phase).
 * Every image is an independent instance of the model problem (Section 3) solved by
 * Algorithm 1 with its own fidelity, alpha, c1, c2 and outer steps; all images share
 * the subdomain size, the number of inner iterations and the initial inner steps, and
 * advance by the same number of outer iterations.  One outer iteration of the whole
 * batch is two kernel launches (multiplier update of every interface of every image,
 * then the local solves of every subdomain of every image: by default a persistent
 * kernel whose clusters walk the batch's work list of (image, subdomain) pairs with
 * each image's fidelity and parameters).  dd_tv_batch_iterate(b, n) with n > 1 is one
 * CUDA-graph launch of the n outer iterations (the graph is captured on the first call
 * with that n and start parity and replayed by later ones).
 * Image sides must be multiples of the subdomain side (64 or 128).  Results are
 * bit-identical to solving each image alone with the same parameters. */
typedef struct dd_tv_batch dd_tv_batch;

typedef struct {
  int height, width;      /* multiples of the subdomain side                           */
  int fidelity;           /* DD_TV_L2, DD_TV_L1 or DD_TV_SEG (no inpainting mask)        */
  double alpha, c1, c2;   /* as in dd_tv_params                                        */
  double tau, sigma;      /* outer steps; tau <= 0 selects Section 5's defaults: tau = 50
                             (1 for DD_TV_SEG), sigma = 1/(2 tau); gamma = 1/(8 tau)      */
} dd_tv_batch_image;

typedef struct {
  int tile;               /* subdomain side: 128 (persistent clusters over the work
                             list, see variant) or 64 (one CTA per subdomain); other
                             sides return DD_TV_EUNSUPPORTED                            */
  int inner_iters;        /* 1..DD_TV_MAX_INNER                                        */
  double tau0, sigma0;    /* initial inner steps (Section 5: 10 and 1/80)               */
  int variant;            /* 0: 4 x 4 pixel micro-tiles per thread (2 x 4 when
                             inner_iters > 64); 2 (tile 128 only): 2 x 4 micro-tiles.
                             Both give the same bits; anything else: DD_TV_EINVAL      */
} dd_tv_batch_params;

/* Validates and allocates the batch (images[n], n >= 1); *out = NULL on error. */
int dd_tv_batch_create(dd_tv_batch** out, const dd_tv_batch_image* images, int n, const dd_tv_batch_params* p);
int dd_tv_batch_destroy(dd_tv_batch* b);                       /* NULL-safe */
const char* dd_tv_batch_last_error(const dd_tv_batch* b);
int dd_tv_batch_set_stream(dd_tv_batch* b, void* stream);
/* Copies f_dev[i] (device, H_i x W_i float32) of every image and initialises every state
 * as dd_tv_load does. */
int dd_tv_batch_load(dd_tv_batch* b, const float* const* f_dev);
/* n_outer outer iterations of every image (asynchronous). */
int dd_tv_batch_iterate(dd_tv_batch* b, int n_outer);
/* Copies image i's current u to u_dev; J(u) of image i (synchronous). */
int dd_tv_batch_get_u(dd_tv_batch* b, int i, float* u_dev);
int dd_tv_batch_energy(dd_tv_batch* b, int i, double* J_out);
/* Total pixels of the batch (sum of H_i W_i). */
long long dd_tv_batch_pixels(const dd_tv_batch* b);

/* ---- Differentiation of the unrolled outer iterations (reverse mode).
 * The paper does not differentiate its method.  These calls give the derivative of
 * u_N, the iterate after N outer iterations of Algorithm 1 from the initial state of
 * dd_tv_load (u^0 = f, 0 on D, or 1/2 for DD_TV_SEG; p~ = 0; lambda = 0), with
 * respect to the data f and the fidelity weight alpha, for a loss L(u_N) whose
 * gradient dL/du_N the caller supplies.  It is the exact derivative of the iteration
 * the solver runs (float32 arithmetic), with the derivative at the kinks of the
 * pointwise maps fixed as: projection onto [-1, 1] passes iff -1 <= t <= 1; the L1
 * shrink passes ubar iff |ubar - f| > sigma_k alpha (else the derivative goes to f);
 * the segmentation clamp passes iff 0 <= x <= 1.  Handles of the decomposed paths
 * (DD_TV_PATH_FUSED, DD_TV_PATH_PLAIN) only; the full-dimension path returns
 * DD_TV_EUNSUPPORTED.
 *
 * dd_tv_adjoint_forward loads f_dev / mask_dev (device, as dd_tv_load; mask nullable)
 * and runs n_outer >= 0 outer iterations, storing the state (u, p~, lambda and the
 * interface values of p~^{n-1}) before every checkpoint_every-th outer iteration in
 * handle-owned device memory: ceil(n_outer / m) + m states of about
 * 4 (3 H W + 5 (interface edges)) bytes each (m = min(checkpoint_every, n_outer)),
 * plus the reverse pass's tape and adjoint fields (about (4 + 2) inner_iters + 60
 * bytes per pixel), allocated on the first call and kept (and grown) until
 * dd_tv_adjoint_release or dd_tv_destroy.  Writes u_N to u_dev (device, H x W).
 * Asynchronous on the handle's stream.  checkpoint_every < 1 returns DD_TV_EINVAL.
 *
 * dd_tv_adjoint_backward reads grad_u_dev (dL/du_N, device H x W) and writes dL/df to
 * grad_f_dev (device H x W; exactly 0 on the inpainting domain D, where nothing
 * depends on f) and dL/dalpha to *grad_alpha (host).  It recomputes each segment of checkpoint_every outer
 * iterations from its checkpoint and then runs the reverse of every outer iteration
 * of the segment, last to first.  The checkpoints stay valid, so it may be called
 * again with another gradient; the handle's current iterate afterwards is
 * unspecified (dd_tv_get_u / dd_tv_iterate need a new load).  Returns DD_TV_EINVAL if
 * no dd_tv_adjoint_forward preceded it since the last load.  Synchronous (it reads
 * the alpha derivative back).
 *
 * dd_tv_set_alpha changes the fidelity weight of an existing handle (same checks as
 * dd_tv_create); the next dd_tv_adjoint_forward / dd_tv_iterate use it.  A changed
 * alpha invalidates the checkpoints of an earlier dd_tv_adjoint_forward: the next
 * dd_tv_adjoint_backward returns DD_TV_EINVAL until a new forward pass is run.
 * dd_tv_adjoint_release frees the checkpoint, tape and adjoint memory. */
int dd_tv_adjoint_forward(dd_tv* h, const float* f_dev, const uint8_t* mask_dev, int n_outer, int checkpoint_every,
                          float* u_dev);
int dd_tv_adjoint_backward(dd_tv* h, const float* grad_u_dev, float* grad_f_dev, double* grad_alpha);
int dd_tv_adjoint_release(dd_tv* h);
int dd_tv_set_alpha(dd_tv* h, double alpha);

#ifdef __cplusplus
}
#endif

#endif /* DD_TV_H */
