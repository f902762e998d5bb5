/*
 * FP64 CPU oracle for the primal-dual domain decomposition method for dual TV
 * minimisation (Lee & Park, "A finite element nonoverlapping domain decomposition
 * method with Lagrange multipliers for the dual total variation minimizations").
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may call, link or load
 * this file; only the test suite, the smoke check and the CPU-baseline leg of the
 * benchmark do.  It shares no code, header, table or constant with the CUDA
 * library: it is a plain, slow, obviously correct restatement of the paper.
 *
 * Conventions (all arrays row-major, double):
 *   image u, f          H x W, pixel (i, j) = row i, column j (Section 2.3)
 *   subdomain grid      NR x NC rectangles; tile row a covers rows
 *                       [floor(a*H/NR), floor((a+1)*H/NR)), tile column b likewise
 *   dual field Y        lowest-order Raviart-Thomas: one dof per pixel edge, the
 *                       normal component, oriented down (p1, horizontal edges) and
 *                       right (p2, vertical edges) (Section 2.3)
 *   global Y arrays     p1 (H+1) x W (edge k is above row k), p2 H x (W+1);
 *                       dofs on the image boundary are 0 (H_0(div))
 *   torn Y~ arrays      every tile keeps its own copy of the dofs on its four sides
 *                       (Section 2.4): P1 has (H+NR) rows x W, tile row a owning
 *                       rows r0(a)+a .. r0(a+1)+a; P2 has H rows x (W+NC) columns,
 *                       tile column b owning columns c0(b)+b .. c0(b+1)+b.
 *                       Sides on the image boundary stay 0; sides on the interface
 *                       Gamma are free dofs.
 *   multipliers         lamh (NR-1) x W: edge between tile rows a, a+1 at column j;
 *                       lamv (NC-1) x H: edge between tile columns b, b+1 at row i.
 *   jump B (Section 2.4) (B p)_e = p_s(e) - p_t(e), s the upper/left tile, t the
 *                       lower/right one (s < t in row-major order, n_st from s to t).
 *
 * Floating point: build with -ffp-contract=off so that x86 and Arm agree.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#define ORC_L2 0  /* F = 1/2 ||A u - f||^2       (ROF, L2 inpainting)  */
#define ORC_L1 1  /* F = ||A u - f||_1           (TV-L1, L1 inpainting) */
#define ORC_SEG 2 /* F = <u, g> + chi_[0,1](u)   (convex Chan-Vese)     */

typedef struct {
  int H, W;        /* image rows, columns                                  */
  int NR, NC;      /* subdomain grid                                       */
  int fidelity;    /* ORC_L2, ORC_L1, ORC_SEG                              */
  double alpha;    /* fidelity weight, > 0                                 */
  double c1, c2;   /* segmentation region constants                       */
  double tau;      /* outer step tau of Algorithm 1                        */
  double sigma;    /* outer step sigma of Algorithm 1                      */
  double tau0;     /* inner initial tau_0 (step on the dual field p)       */
  double sigma0;   /* inner initial sigma_0 (step on the image u)          */
  double gamma;    /* inner acceleration parameter gamma                   */
  int inner;       /* inner iterations per outer iteration                 */
} orc_params;

/* ---------------------------------------------------------------- partition */

static int part_start(int a, int len, int n) { return (int)(((long long)a * len) / n); }

/* ----------------------------------------------------------- compensated sum */

typedef struct { double s, c; } nsum; /* Neumaier's improved Kahan summation */

static void nsum_add(nsum* acc, double x) {
  double t = acc->s + x;
  if (fabs(acc->s) >= fabs(x)) acc->c += (acc->s - t) + x;
  else acc->c += (x - t) + acc->s;
  acc->s = t;
}
static double nsum_get(const nsum* acc) { return acc->s + acc->c; }

/* ------------------------------------------------ pointwise maps (Section 3) */

/* shrinkage shr(v, s) = max(|v| - s, 0) v / |v|, with 0/|0| = 0 (eq. shrinkage) */
static double shrink(double v, double s) {
  double m = fabs(v) - s;
  if (m <= 0.0) return 0.0;
  return v > 0.0 ? m : -m;
}

/* prox_{s F} at one pixel, s = sigma_0 * alpha (Section 3 and Section 5.1-5.3):
 *   L2 : (v + s f) / (1 + s) off D, v on D
 *   L1 : f + shr(v - f, s)      off D, v on D
 *   SEG: proj_[0,1](v - s g),  g = (f - c1)^2 - (f - c2)^2            */
static double prox_pixel(int fid, double v, double f, int in_d, double s, double c1, double c2) {
  if (fid == ORC_SEG) {
    double g = (f - c1) * (f - c1) - (f - c2) * (f - c2);
    double x = v - s * g;
    return x < 0.0 ? 0.0 : (x > 1.0 ? 1.0 : x);
  }
  if (in_d) return v;
  if (fid == ORC_L2) return (v + s * f) / (1.0 + s);
  return f + shrink(v - f, s);
}

/* projection onto [-1, 1] (eq. proj_C) */
static double clamp1(double x) { return x / (fabs(x) > 1.0 ? fabs(x) : 1.0); }

void orc_prox(int fid, int n, const double* v, const double* f, const unsigned char* mask,
              double s, double c1, double c2, double* out) {
  for (int k = 0; k < n; ++k) out[k] = prox_pixel(fid, v[k], f[k], mask ? mask[k] : 0, s, c1, c2);
}

/* ------------------------------------- global operators on Y (Section 2.3) */

/* div p on the whole image: p1 (H+1) x W, p2 H x (W+1) */
void orc_div(int H, int W, const double* p1, const double* p2, double* out) {
  for (int i = 0; i < H; ++i)
    for (int j = 0; j < W; ++j)
      out[i * W + j] = p1[(i + 1) * W + j] - p1[i * W + j] + p2[i * (W + 1) + j + 1] - p2[i * (W + 1) + j];
}

/* D u = -div^* u on the interior edges (forward differences, eq. FFD); the image
 * boundary edges are not dofs of Y and get 0. */
void orc_grad(int H, int W, const double* u, double* g1, double* g2) {
  for (int k = 0; k <= H; ++k)
    for (int j = 0; j < W; ++j)
      g1[k * W + j] = (k == 0 || k == H) ? 0.0 : u[k * W + j] - u[(k - 1) * W + j];
  for (int i = 0; i < H; ++i)
    for (int l = 0; l <= W; ++l)
      g2[i * (W + 1) + l] = (l == 0 || l == W) ? 0.0 : u[i * W + l] - u[i * W + l - 1];
}

/* ------------------------------------------------ energies (Section 3, 5) */

/* anisotropic TV(u) = sum |u_{i+1,j} - u_ij| + |u_{i,j+1} - u_ij| (Proposition on
 * the FE/FD equivalence, eq. FFD), compensated sum */
double orc_tv(int H, int W, const double* u) {
  nsum acc = {0.0, 0.0};
  for (int i = 0; i < H; ++i)
    for (int j = 0; j < W; ++j) {
      if (i + 1 < H) nsum_add(&acc, fabs(u[(i + 1) * W + j] - u[i * W + j]));
      if (j + 1 < W) nsum_add(&acc, fabs(u[i * W + j + 1] - u[i * W + j]));
    }
  return nsum_get(&acc);
}

/* F(u) for the three fidelities; +inf for SEG when u leaves [0, 1] */
double orc_fidelity(int fid, int n, const double* u, const double* f, const unsigned char* mask,
                    double c1, double c2) {
  nsum acc = {0.0, 0.0};
  for (int k = 0; k < n; ++k) {
    if (fid == ORC_SEG) {
      if (u[k] < 0.0 || u[k] > 1.0) return INFINITY;
      double g = (f[k] - c1) * (f[k] - c1) - (f[k] - c2) * (f[k] - c2);
      nsum_add(&acc, u[k] * g);
      continue;
    }
    if (mask && mask[k]) continue;
    double r = u[k] - f[k];
    nsum_add(&acc, fid == ORC_L2 ? 0.5 * r * r : fabs(r));
  }
  return nsum_get(&acc);
}

/* J(u) = alpha F(u) + TV(u) (eq. model) */
double orc_energy(const orc_params* pr, const double* u, const double* f, const unsigned char* mask) {
  return pr->alpha * orc_fidelity(pr->fidelity, pr->H * pr->W, u, f, mask, pr->c1, pr->c2) +
         orc_tv(pr->H, pr->W, u);
}

/* Dual value of a global p in C (Fenchel-Rockafellar dual of eq. model, with the
 * conjugate scaled as alpha F^*(div p / alpha)):
 *   L2 (no mask): -(1/(2 alpha)) ||div p + alpha f||^2 + (alpha/2) ||f||^2
 *   SEG         : sum_T min(0, (alpha g - div p)_T)
 *   L1 (no mask): -<f, div p>, after p is scaled by min(1, alpha / ||div p||_inf)
 * Weak duality gives d(p) <= J(u) for every u.  Masked problems have no finite
 * certificate here and return -inf. */
double orc_dual_value(const orc_params* pr, const double* p1, const double* p2, const double* f,
                      const unsigned char* mask) {
  int H = pr->H, W = pr->W, n = H * W;
  double a = pr->alpha, out = -INFINITY;
  if (pr->fidelity != ORC_SEG && mask)
    for (int k = 0; k < n; ++k)
      if (mask[k]) return -INFINITY;
  double* d = (double*)malloc(sizeof(double) * n);
  orc_div(H, W, p1, p2, d);
  nsum acc = {0.0, 0.0};
  if (pr->fidelity == ORC_SEG) {
    for (int k = 0; k < n; ++k) {
      double g = (f[k] - pr->c1) * (f[k] - pr->c1) - (f[k] - pr->c2) * (f[k] - pr->c2);
      double t = a * g - d[k];
      nsum_add(&acc, t < 0.0 ? t : 0.0);
    }
    out = nsum_get(&acc);
  } else if (pr->fidelity == ORC_L2) {
    for (int k = 0; k < n; ++k) {
      double t = d[k] + a * f[k];
      nsum_add(&acc, -t * t / (2.0 * a) + 0.5 * a * f[k] * f[k]);
    }
    out = nsum_get(&acc);
  } else {
    double dmax = 0.0;
    for (int k = 0; k < n; ++k) dmax = fabs(d[k]) > dmax ? fabs(d[k]) : dmax;
    double scale = dmax > a ? a / dmax : 1.0;
    for (int k = 0; k < n; ++k) nsum_add(&acc, -f[k] * scale * d[k]);
    out = nsum_get(&acc);
  }
  free(d);
  return out;
}

/* ------------------------------------------- torn space and jump (Section 2.4) */

/* (B p~) on every interface dof.  jh (NR-1) x W, jv (NC-1) x H. */
void orc_jump(const orc_params* pr, const double* P1, const double* P2, double* jh, double* jv) {
  int H = pr->H, W = pr->W, W2 = W + pr->NC;
  for (int a = 0; a + 1 < pr->NR; ++a) {
    int rs = part_start(a + 1, H, pr->NR) + a; /* bottom side of tile row a   */
    int rt = rs + 1;                           /* top side of tile row a + 1  */
    for (int j = 0; j < W; ++j) jh[a * W + j] = P1[rs * W + j] - P1[rt * W + j];
  }
  for (int b = 0; b + 1 < pr->NC; ++b) {
    int cs = part_start(b + 1, W, pr->NC) + b; /* right side of tile column b  */
    int ct = cs + 1;                           /* left side of tile column b+1 */
    for (int i = 0; i < H; ++i) jv[b * H + i] = P2[i * W2 + cs] - P2[i * W2 + ct];
  }
}

/* B^* lambda: +lambda_e on the s-side copy, -lambda_e on the t-side copy, 0 elsewhere. */
void orc_jump_adjoint(const orc_params* pr, const double* lamh, const double* lamv, double* P1, double* P2) {
  int H = pr->H, W = pr->W, W2 = W + pr->NC;
  memset(P1, 0, sizeof(double) * (size_t)(H + pr->NR) * W);
  memset(P2, 0, sizeof(double) * (size_t)H * W2);
  for (int a = 0; a + 1 < pr->NR; ++a) {
    int rs = part_start(a + 1, H, pr->NR) + a, rt = rs + 1;
    for (int j = 0; j < W; ++j) {
      P1[rs * W + j] += lamh[a * W + j];
      P1[rt * W + j] -= lamh[a * W + j];
    }
  }
  for (int b = 0; b + 1 < pr->NC; ++b) {
    int cs = part_start(b + 1, W, pr->NC) + b, ct = cs + 1;
    for (int i = 0; i < H; ++i) {
      P2[i * W2 + cs] += lamv[b * H + i];
      P2[i * W2 + ct] -= lamv[b * H + i];
    }
  }
}

/* ---------------------------------------- local operators on one tile */

typedef struct {
  int mr, mc;                     /* tile rows, columns                     */
  int top, bottom, left, right;   /* 1 if that side lies on Gamma (active)  */
} orc_tile;

/* div_s p on the tile: p1 (mr+1) x mc, p2 mr x (mc+1) */
static void tile_div(const orc_tile* t, const double* p1, const double* p2, double* out) {
  int mr = t->mr, mc = t->mc;
  for (int i = 0; i < mr; ++i)
    for (int j = 0; j < mc; ++j)
      out[i * mc + j] = p1[(i + 1) * mc + j] - p1[i * mc + j] + p2[i * (mc + 1) + j + 1] - p2[i * (mc + 1) + j];
}

/* D_s u = -div_s^* u on the tile's dofs; pixels outside the tile count as 0, and
 * sides on the image boundary are not dofs (returned as 0). */
static void tile_grad(const orc_tile* t, const double* u, double* g1, double* g2) {
  int mr = t->mr, mc = t->mc;
  for (int k = 0; k <= mr; ++k)
    for (int j = 0; j < mc; ++j) {
      double below = k < mr ? u[k * mc + j] : 0.0;
      double above = k > 0 ? u[(k - 1) * mc + j] : 0.0;
      int active = (k > 0 && k < mr) || (k == 0 && t->top) || (k == mr && t->bottom);
      g1[k * mc + j] = active ? below - above : 0.0;
    }
  for (int i = 0; i < mr; ++i)
    for (int l = 0; l <= mc; ++l) {
      double right = l < mc ? u[i * mc + l] : 0.0;
      double left = l > 0 ? u[i * mc + l - 1] : 0.0;
      int active = (l > 0 && l < mc) || (l == 0 && t->left) || (l == mc && t->right);
      g2[i * (mc + 1) + l] = active ? right - left : 0.0;
    }
}

void orc_tile_div(int mr, int mc, const double* p1, const double* p2, double* out) {
  orc_tile t = {mr, mc, 1, 1, 1, 1};
  tile_div(&t, p1, p2, out);
}

void orc_tile_grad(int mr, int mc, int top, int bottom, int left, int right, const double* u, double* g1,
                   double* g2) {
  orc_tile t = {mr, mc, top, bottom, left, right};
  tile_grad(&t, u, g1, g2);
}

/* Relative change of the dual field over one inner iteration, the quantity of the
 * inner stopping rule (Section 5, eq. stop_inner1):
 *   ||p^{k+1} - p^k||_2 / ||p^{k+1}||_2   over the tile's active dofs;
 * 0 when p^{k+1} = 0 (nothing left to change: the rule counts it as converged). */
static double rel_change(const orc_tile* t, const double* p1_new, const double* p2_new, const double* p1_old,
                         const double* p2_old) {
  int mr = t->mr, mc = t->mc;
  nsum dd = {0.0, 0.0}, pp = {0.0, 0.0};
  for (int e = 0; e < (mr + 1) * mc; ++e) {
    nsum_add(&dd, (p1_new[e] - p1_old[e]) * (p1_new[e] - p1_old[e]));
    nsum_add(&pp, p1_new[e] * p1_new[e]);
  }
  for (int e = 0; e < mr * (mc + 1); ++e) {
    nsum_add(&dd, (p2_new[e] - p2_old[e]) * (p2_new[e] - p2_old[e]));
    nsum_add(&pp, p2_new[e] * p2_new[e]);
  }
  double num = nsum_get(&dd), den = nsum_get(&pp);
  return den > 0.0 ? sqrt(num / den) : 0.0;
}

/* Local solver (Section 5, local problem eq. local): accelerated primal-dual
 * iteration (Chambolle-Pock, Algorithm 2 of their 2011 paper) on
 *   min_u max_p  -<u, div_s p> + alpha F_s(u) - G_s^*(p),
 *   G_s^*(p) = chi_C(p) + (1/(2 tau)) ||p - phat||^2,
 * where G_s^* is (1/tau)-uniformly convex, so the dual field p plays the role of
 * the accelerated variable.  One iteration, with steps (tau_k on p, sigma_k on u):
 *   u    <- prox_{sigma_k alpha F}(u + sigma_k div_s pbar)
 *   pnew <- proj_C((tau (p + tau_k D_s u) + tau_k phat) / (tau + tau_k))
 *   theta = 1 / sqrt(1 + 2 gamma tau_k);  tau_{k+1} = theta tau_k;  sigma_{k+1} = sigma_k / theta
 *   pbar <- pnew + theta (pnew - p);  p <- pnew
 * The schedule restarts at (tau0, sigma0) and pbar = p at every call.
 * phat == NULL selects the plain single-domain step (no proximal term, used by
 * the N = 1 comparator).  f, mask, u are the tile's pixels (mr x mc).
 * tol > 0: stop after the first iteration whose relative change of p (rel_change)
 * is below tol, at most iters iterations (eq. stop_inner1); res (nullable, iters
 * entries) receives the relative change of every iteration run.  Returns the number
 * of iterations run. */
static int local_solve(const orc_params* pr, const orc_tile* t, const double* f, const unsigned char* mask,
                       double* u, double* p1, double* p2, const double* ph1, const double* ph2, int iters,
                       double tol, double* res) {
  int mr = t->mr, mc = t->mc;
  int n1 = (mr + 1) * mc, n2 = mr * (mc + 1), np = mr * mc;
  double* pb1 = (double*)malloc(sizeof(double) * n1);
  double* pb2 = (double*)malloc(sizeof(double) * n2);
  double* d = (double*)malloc(sizeof(double) * np);
  double* g1 = (double*)malloc(sizeof(double) * n1);
  double* g2 = (double*)malloc(sizeof(double) * n2);
  double* o1 = (tol > 0.0 || res) ? (double*)malloc(sizeof(double) * n1) : NULL;
  double* o2 = (tol > 0.0 || res) ? (double*)malloc(sizeof(double) * n2) : NULL;
  memcpy(pb1, p1, sizeof(double) * n1);
  memcpy(pb2, p2, sizeof(double) * n2);
  double tk = pr->tau0, sk = pr->sigma0, tau = pr->tau;
  int done = 0;
  for (int k = 0; k < iters; ++k) {
    if (o1) {
      memcpy(o1, p1, sizeof(double) * n1);
      memcpy(o2, p2, sizeof(double) * n2);
    }
    /* u-step */
    tile_div(t, pb1, pb2, d);
    for (int q = 0; q < np; ++q)
      u[q] = prox_pixel(pr->fidelity, u[q] + sk * d[q], f[q], mask ? mask[q] : 0, sk * pr->alpha, pr->c1, pr->c2);
    /* p-step; inactive sides have g = 0 and p = 0 and stay 0 */
    tile_grad(t, u, g1, g2);
    double theta = 1.0 / sqrt(1.0 + 2.0 * pr->gamma * tk);
    for (int e = 0; e < n1; ++e) {
      int kk = e / mc;
      int active = (kk > 0 && kk < mr) || (kk == 0 && t->top) || (kk == mr && t->bottom);
      if (!active) continue;
      double q = p1[e] + tk * g1[e];
      double pn = ph1 ? clamp1((tau * q + tk * ph1[e]) / (tau + tk)) : clamp1(q);
      pb1[e] = pn + theta * (pn - p1[e]);
      p1[e] = pn;
    }
    for (int e = 0; e < n2; ++e) {
      int l = e % (mc + 1);
      int active = (l > 0 && l < mc) || (l == 0 && t->left) || (l == mc && t->right);
      if (!active) continue;
      double q = p2[e] + tk * g2[e];
      double pn = ph2 ? clamp1((tau * q + tk * ph2[e]) / (tau + tk)) : clamp1(q);
      pb2[e] = pn + theta * (pn - p2[e]);
      p2[e] = pn;
    }
    tk = theta * tk;
    sk = sk / theta;
    done = k + 1;
    if (o1) {
      double rc = rel_change(t, p1, p2, o1, o2);
      if (res) res[k] = rc;
      if (tol > 0.0 && rc < tol) break;
    }
  }
  free(pb1); free(pb2); free(d); free(g1); free(g2); free(o1); free(o2);
  return done;
}

/* extract / store one tile's block of the torn arrays */
static void tile_geometry(const orc_params* pr, int a, int b, orc_tile* t, int* r0, int* c0) {
  *r0 = part_start(a, pr->H, pr->NR);
  *c0 = part_start(b, pr->W, pr->NC);
  t->mr = part_start(a + 1, pr->H, pr->NR) - *r0;
  t->mc = part_start(b + 1, pr->W, pr->NC) - *c0;
  t->top = a > 0;
  t->bottom = a + 1 < pr->NR;
  t->left = b > 0;
  t->right = b + 1 < pr->NC;
}

static void gather_tile(const orc_params* pr, int a, int b, const orc_tile* t, int r0, int c0, const double* img,
                        const double* P1, const double* P2, double* ls, double* l1, double* l2) {
  int W = pr->W, W2 = W + pr->NC, mr = t->mr, mc = t->mc;
  if (img)
    for (int i = 0; i < mr; ++i)
      for (int j = 0; j < mc; ++j) ls[i * mc + j] = img[(r0 + i) * W + c0 + j];
  if (P1)
    for (int k = 0; k <= mr; ++k)
      for (int j = 0; j < mc; ++j) l1[k * mc + j] = P1[(r0 + a + k) * W + c0 + j];
  if (P2)
    for (int i = 0; i < mr; ++i)
      for (int l = 0; l <= mc; ++l) l2[i * (mc + 1) + l] = P2[(r0 + i) * W2 + c0 + b + l];
}

static void scatter_tile(const orc_params* pr, int a, int b, const orc_tile* t, int r0, int c0, double* img,
                         double* P1, double* P2, const double* ls, const double* l1, const double* l2) {
  int W = pr->W, W2 = W + pr->NC, mr = t->mr, mc = t->mc;
  for (int i = 0; i < mr; ++i)
    for (int j = 0; j < mc; ++j) img[(r0 + i) * W + c0 + j] = ls[i * mc + j];
  for (int k = 0; k <= mr; ++k)
    for (int j = 0; j < mc; ++j) P1[(r0 + a + k) * W + c0 + j] = l1[k * mc + j];
  for (int i = 0; i < mr; ++i)
    for (int l = 0; l <= mc; ++l) P2[(r0 + i) * W2 + c0 + b + l] = l2[i * (mc + 1) + l];
}

/* -------------------------------------------------------------- Algorithm 1 */

/* Runs n_outer iterations of Algorithm 1 on the state (u, P1, P2, P1prev, P2prev,
 * lamh, lamv), all in/out:
 *   lambda^{n+1} = lambda^n + sigma B (2 p~^n - p~^{n-1})
 *   phat^{n+1}   = p~^n - tau B^* lambda^{n+1}
 *   for every tile s, in parallel: (u_s, p~_s) <- local solve warm-started from
 *                  (u_s^n, p~_s^n) with proximal centre phat^{n+1}|_s
 *   p~^{n-1} <- p~^n, then u^{n+1}, p~^{n+1} are the assembled local results.
 * energy_trace (nullable) receives J(u^{n+1}) after every outer iteration.
 * mask (nullable) marks the inpainting domain D (1 = in D).  Returns 0. */
/* orc_dd_run_ex: the same with the inner count of every local solve under control:
 *   inner_tol > 0      adaptive inner stopping (eq. stop_inner1), at most pr->inner;
 *   counts_in != NULL  tile s of outer iteration n runs exactly counts_in[n T + s]
 *                      iterations (T = NR NC; overrides inner_tol);
 *   counts_out, res    (nullable) receive the iterations run, n_outer x T, and the
 *                      relative change of p of every iteration, n_outer x T x pr->inner
 *                      (entries past the last iteration are left untouched). */
int orc_dd_run_ex(const orc_params* pr, const double* f, const unsigned char* mask, int n_outer, double inner_tol,
                  const int* counts_in, int* counts_out, double* res, double* u, double* P1, double* P2,
                  double* P1prev, double* P2prev, double* lamh, double* lamv, double* energy_trace);

int orc_dd_run(const orc_params* pr, const double* f, const unsigned char* mask, int n_outer, double* u,
               double* P1, double* P2, double* P1prev, double* P2prev, double* lamh, double* lamv,
               double* energy_trace) {
  return orc_dd_run_ex(pr, f, mask, n_outer, 0.0, NULL, NULL, NULL, u, P1, P2, P1prev, P2prev, lamh, lamv,
                       energy_trace);
}

int orc_dd_run_ex(const orc_params* pr, const double* f, const unsigned char* mask, int n_outer, double inner_tol,
                  const int* counts_in, int* counts_out, double* res, double* u, double* P1, double* P2,
                  double* P1prev, double* P2prev, double* lamh, double* lamv, double* energy_trace) {
  int H = pr->H, W = pr->W, NR = pr->NR, NC = pr->NC;
  size_t n1 = (size_t)(H + NR) * W, n2 = (size_t)H * (W + NC);
  size_t nh = (size_t)(NR - 1) * W, nv = (size_t)(NC - 1) * H;
  double* jh = (double*)malloc(sizeof(double) * (nh ? nh : 1));
  double* jv = (double*)malloc(sizeof(double) * (nv ? nv : 1));
  double* jh_prev = (double*)malloc(sizeof(double) * (nh ? nh : 1));
  double* jv_prev = (double*)malloc(sizeof(double) * (nv ? nv : 1));
  double* Ph1 = (double*)malloc(sizeof(double) * n1);
  double* Ph2 = (double*)malloc(sizeof(double) * n2);
  for (int n = 0; n < n_outer; ++n) {
    /* multiplier update */
    orc_jump(pr, P1, P2, jh, jv);
    orc_jump(pr, P1prev, P2prev, jh_prev, jv_prev);
    for (size_t e = 0; e < nh; ++e) lamh[e] += pr->sigma * (2.0 * jh[e] - jh_prev[e]);
    for (size_t e = 0; e < nv; ++e) lamv[e] += pr->sigma * (2.0 * jv[e] - jv_prev[e]);
    /* proximal centre phat = p~^n - tau B^* lambda^{n+1} */
    orc_jump_adjoint(pr, lamh, lamv, Ph1, Ph2);
    for (size_t e = 0; e < n1; ++e) Ph1[e] = P1[e] - pr->tau * Ph1[e];
    for (size_t e = 0; e < n2; ++e) Ph2[e] = P2[e] - pr->tau * Ph2[e];
    /* keep p~^n as the next "previous" iterate */
    memcpy(P1prev, P1, sizeof(double) * n1);
    memcpy(P2prev, P2, sizeof(double) * n2);
    /* local solves, one per tile, in parallel */
#pragma omp parallel for schedule(dynamic)
    for (int s = 0; s < NR * NC; ++s) {
      int a = s / NC, b = s % NC, r0, c0;
      orc_tile t;
      tile_geometry(pr, a, b, &t, &r0, &c0);
      int np = t.mr * t.mc, l1n = (t.mr + 1) * t.mc, l2n = t.mr * (t.mc + 1);
      double* lu = (double*)malloc(sizeof(double) * np);
      double* lf = (double*)malloc(sizeof(double) * np);
      unsigned char* lm = NULL;
      double* lp1 = (double*)malloc(sizeof(double) * l1n);
      double* lp2 = (double*)malloc(sizeof(double) * l2n);
      double* lh1 = (double*)malloc(sizeof(double) * l1n);
      double* lh2 = (double*)malloc(sizeof(double) * l2n);
      gather_tile(pr, a, b, &t, r0, c0, u, P1, P2, lu, lp1, lp2);
      gather_tile(pr, a, b, &t, r0, c0, f, Ph1, Ph2, lf, lh1, lh2);
      if (mask) {
        lm = (unsigned char*)malloc(np);
        for (int i = 0; i < t.mr; ++i)
          for (int j = 0; j < t.mc; ++j) lm[i * t.mc + j] = mask[(r0 + i) * W + c0 + j];
      }
      const size_t slot = (size_t)n * NR * NC + s;
      const int iters = counts_in ? counts_in[slot] : pr->inner;
      const double tol = counts_in ? 0.0 : inner_tol;
      const int ran = local_solve(pr, &t, lf, lm, lu, lp1, lp2, lh1, lh2, iters, tol,
                                  res ? res + slot * pr->inner : NULL);
      if (counts_out) counts_out[slot] = ran;
      scatter_tile(pr, a, b, &t, r0, c0, u, P1, P2, lu, lp1, lp2);
      free(lu); free(lf); free(lm); free(lp1); free(lp2); free(lh1); free(lh2);
    }
    if (energy_trace) energy_trace[n] = orc_energy(pr, u, f, mask);
  }
  free(jh); free(jv); free(jh_prev); free(jv_prev); free(Ph1); free(Ph2);
  return 0;
}

/* One local solve on a single tile, exposed for the tests (in/out u, p1, p2). */
void orc_local_solve(const orc_params* pr, int mr, int mc, int top, int bottom, int left, int right,
                     const double* f, const unsigned char* mask, double* u, double* p1, double* p2,
                     const double* ph1, const double* ph2, int iters) {
  orc_tile t = {mr, mc, top, bottom, left, right};
  local_solve(pr, &t, f, mask, u, p1, p2, ph1, ph2, iters, 0.0, NULL);
}

/* ------------------------------------------- full-dimension comparators */

/* Plain primal-dual iteration on the undecomposed problem (the N = 1 comparator
 * of Section 5): constant steps tau0 on p and sigma0 on u, theta = 1.
 *   u    <- prox_{sigma0 alpha F}(u + sigma0 div pbar)
 *   pnew <- proj_C(p + tau0 D u);  pbar <- 2 pnew - p;  p <- pnew
 * State in/out: u (H x W), p1, p2, pb1, pb2 (global Y layout). */
int orc_cp_run(const orc_params* pr, const double* f, const unsigned char* mask, int iters, double* u, double* p1,
               double* p2, double* pb1, double* pb2) {
  int H = pr->H, W = pr->W;
  size_t n1 = (size_t)(H + 1) * W, n2 = (size_t)H * (W + 1), np = (size_t)H * W;
  double* d = (double*)malloc(sizeof(double) * np);
  double* g1 = (double*)malloc(sizeof(double) * n1);
  double* g2 = (double*)malloc(sizeof(double) * n2);
  double s = pr->sigma0, t = pr->tau0;
  for (int k = 0; k < iters; ++k) {
    orc_div(H, W, pb1, pb2, d);
#pragma omp parallel for
    for (int i = 0; i < H; ++i)
      for (int j = 0; j < W; ++j) {
        size_t q = (size_t)i * W + j;
        u[q] = prox_pixel(pr->fidelity, u[q] + s * d[q], f[q], mask ? mask[q] : 0, s * pr->alpha, pr->c1, pr->c2);
      }
    orc_grad(H, W, u, g1, g2);
#pragma omp parallel for
    for (int k1 = 1; k1 < H; ++k1)
      for (int j = 0; j < W; ++j) {
        size_t e = (size_t)k1 * W + j;
        double pn = clamp1(p1[e] + t * g1[e]);
        pb1[e] = 2.0 * pn - p1[e];
        p1[e] = pn;
      }
#pragma omp parallel for
    for (int i = 0; i < H; ++i)
      for (int l = 1; l < W; ++l) {
        size_t e = (size_t)i * (W + 1) + l;
        double pn = clamp1(p2[e] + t * g2[e]);
        pb2[e] = 2.0 * pn - p2[e];
        p2[e] = pn;
      }
  }
  free(d); free(g1); free(g2);
  return 0;
}

/* Accelerated primal-dual iteration for the unmasked ROF problem, used only to
 * certify a reference minimum J* through the duality gap.  Here the image u is
 * the accelerated variable (alpha F is alpha-strongly convex):
 *   p    <- proj_C(p + s_k D ubar)
 *   unew <- (u + t_k div p + t_k alpha f) / (1 + t_k alpha)
 *   theta = 1 / sqrt(1 + 2 alpha t_k);  t_{k+1} = theta t_k;  s_{k+1} = s_k / theta
 *   ubar <- unew + theta (unew - u);  u <- unew
 * steps[2] = (t_k, s_k) in/out; ubar in/out. */
int orc_rof_accel_run(const orc_params* pr, const double* f, int iters, double* u, double* ubar, double* p1,
                      double* p2, double* steps) {
  int H = pr->H, W = pr->W;
  size_t n1 = (size_t)(H + 1) * W, n2 = (size_t)H * (W + 1), np = (size_t)H * W;
  double* d = (double*)malloc(sizeof(double) * np);
  double* g1 = (double*)malloc(sizeof(double) * n1);
  double* g2 = (double*)malloc(sizeof(double) * n2);
  double t = steps[0], s = steps[1], a = pr->alpha;
  for (int k = 0; k < iters; ++k) {
    orc_grad(H, W, ubar, g1, g2);
#pragma omp parallel for
    for (int k1 = 1; k1 < H; ++k1)
      for (int j = 0; j < W; ++j) {
        size_t e = (size_t)k1 * W + j;
        p1[e] = clamp1(p1[e] + s * g1[e]);
      }
#pragma omp parallel for
    for (int i = 0; i < H; ++i)
      for (int l = 1; l < W; ++l) {
        size_t e = (size_t)i * (W + 1) + l;
        p2[e] = clamp1(p2[e] + s * g2[e]);
      }
    orc_div(H, W, p1, p2, d);
    double theta = 1.0 / sqrt(1.0 + 2.0 * a * t);
#pragma omp parallel for
    for (int i = 0; i < H; ++i)
      for (int j = 0; j < W; ++j) {
        size_t q = (size_t)i * W + j;
        double un = (u[q] + t * d[q] + t * a * f[q]) / (1.0 + t * a);
        ubar[q] = un + theta * (un - u[q]);
        u[q] = un;
      }
    t = theta * t;
    s = s / theta;
  }
  steps[0] = t;
  steps[1] = s;
  free(d); free(g1); free(g2);
  return 0;
}

/* Averages the two copies of every interface dof of a torn field into a global
 * field of Y (the average of two points of the box C stays in C).  Used for the
 * duality-gap certificate of a domain decomposition iterate. */
void orc_torn_to_global(const orc_params* pr, const double* P1, const double* P2, double* p1, double* p2) {
  int H = pr->H, W = pr->W, W2 = W + pr->NC;
  memset(p1, 0, sizeof(double) * (size_t)(H + 1) * W);
  memset(p2, 0, sizeof(double) * (size_t)H * (W + 1));
  for (int a = 0; a < pr->NR; ++a) {
    int r0 = part_start(a, H, pr->NR), r1 = part_start(a + 1, H, pr->NR);
    for (int k = r0; k <= r1; ++k) {
      if (k == 0 || k == H) continue;
      for (int j = 0; j < W; ++j) {
        double v = P1[(k + a) * W + j];
        if (k == r1) v = 0.5 * (v + P1[(k + a + 1) * W + j]); /* s side + t side */
        if (k == r0) continue;                                 /* counted by the tile above */
        p1[k * W + j] = v;
      }
    }
  }
  for (int b = 0; b < pr->NC; ++b) {
    int c0 = part_start(b, W, pr->NC), c1 = part_start(b + 1, W, pr->NC);
    for (int i = 0; i < H; ++i)
      for (int l = c0; l <= c1; ++l) {
        if (l == 0 || l == W || l == c0) continue;
        double v = P2[i * W2 + l + b];
        if (l == c1) v = 0.5 * (v + P2[i * W2 + l + b + 1]);
        p2[i * (W + 1) + l] = v;
      }
  }
}
