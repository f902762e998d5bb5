// Reverse-mode derivative of the unrolled outer iterations of Algorithm 1 with
// respect to the data f and the fidelity weight alpha.  (The paper does not
// differentiate its method; this is the adjoint of exactly the iteration the
// solver runs, with the derivative of each kink fixed as follows: the projection
// onto [-1, 1] passes iff -1 <= t <= 1, the L1 shrink passes ubar iff
// |ubar - f| > sigma_k alpha, the segmentation clamp passes iff 0 <= x <= 1.)
//
// Forward inner iteration k of a local solve (Section 5), per tile, with q = pbar:
//   ubar  = u + sigma_k div q                 u' = prox_{sigma_k alpha F}(ubar)
//   t     = pa p + pc D u' + pb phat          p' = proj_C(t)     (pa, pc, pb of Coef)
//   q'    = p' + theta_k (p' - p)
// Reverse of iteration k, given the adjoints (Au, AP, AQ) of (u', p', q'):
//   at    = [t in C] (AP + (1 + theta_k) AQ)            (0 on inactive dofs)
//   Au'   = Au - div(pc at)                            (D^T = -div on the tile)
//   Aubar = prox'(ubar) Au';   Af += d prox/df Au';   Aalpha += d prox/dalpha Au'
//   Au <- Aubar;  Ad = sigma_k Aubar;  AQ <- -D Ad;  AP <- pa at - theta_k AQ;
//   APhat += pb at.
// The forward values the reverse needs (ubar_k and the projection's pass bit of every
// dof) are recorded by a recomputation of the outer iteration (the tape kernels
// below, which run the plain path's arithmetic bit for bit).  All kernels stream
// whole fields through HBM, one thread per pixel (grid-stride).
#include "internal.cuh"

namespace ddtv {

namespace {

constexpr int kBlock = 256;
constexpr int kBX = 32, kBY = kBlock / kBX;  // per-pixel kernels: 32 columns x 8 rows per block

int nblocks(long long n) {
  long long b = (n + kBlock - 1) / kBlock;
  if (b > 152 * 32) b = 152 * 32;
  return (int)(b < 1 ? 1 : b);
}

dim3 pixel_grid(const Grid& g) { return dim3((g.W + kBX - 1) / kBX, (g.H + kBY - 1) / kBY, 1); }

// One thread per pixel (i, j) of a 2-D grid; the tile row / column of every pixel row
// / column and the tile's first and end rows / columns come from small tables (x = tile
// index, y = first, z = end), so no per-pixel division is needed.
struct Pix {
  int i, j, a, b, r0, r1, c0, c1;
};

__device__ __forceinline__ bool pixel_of(const Grid& g, const int4* __restrict__ rt, const int4* __restrict__ ct,
                                         Pix& p) {
  p.j = blockIdx.x * kBX + threadIdx.x;
  p.i = blockIdx.y * kBY + threadIdx.y;
  if (p.i >= g.H || p.j >= g.W) return false;
  const int4 r = __ldg(rt + p.i), c = __ldg(ct + p.j);
  p.a = r.x;
  p.r0 = r.y;
  p.r1 = r.z;
  p.b = c.x;
  p.c0 = c.y;
  p.c1 = c.z;
  return true;
}

// ---- tape: forward steps that also record what the reverse needs

template <int FID, bool MASK>
__global__ void __launch_bounds__(kBlock) k_ustep_tape(Grid g, const int4* __restrict__ rt,
                                                       const int4* __restrict__ ct, float c1, float c2,
                                                       const float* __restrict__ f, const uint8_t* __restrict__ mask,
                                                       float* __restrict__ u, const float* __restrict__ Pb1,
                                                       const float* __restrict__ Pb2, const Coef* __restrict__ ck,
                                                       float* __restrict__ ubar_out) {
  Pix q;
  if (!pixel_of(g, rt, ct, q)) return;
  const Coef c = *ck;
  const int W2 = g.W + g.NC;
  const size_t px = (size_t)q.i * g.W + q.j;
  const size_t et = (size_t)(q.i + q.a) * g.W + q.j, el = (size_t)q.i * W2 + q.j + q.b;
  const float d = div_px(Pb1[et], Pb1[et + g.W], Pb2[el], Pb2[el + 1]);
  float fv = f[px];
  if (FID == FID_SEG) fv = (fv - c1) * (fv - c1) - (fv - c2) * (fv - c2);
  const bool in_d = MASK && mask[px];
  const float uo = u[px];
  ubar_out[px] = fmaf(c.sig, d, uo);  // the value u_update forms internally
  u[px] = u_update<FID>(uo, d, fv, in_d, c);
}

__device__ __forceinline__ void p_tape_dof(float* __restrict__ P, float* __restrict__ Pb, const float* __restrict__ Ph,
                                           uint8_t* __restrict__ M, size_t e, float du, const Coef& c) {
  float p = P[e], q;
  const float ph = Ph[e];
  const float t = p_target(p, du, ph, c);
  M[e] = (t >= -1.0f && t <= 1.0f) ? 1 : 0;
  p_update(p, q, du, ph, c);
  P[e] = p;
  Pb[e] = q;
}

// p-step over the torn field (same dof ownership as the plain path) recording the
// projection's pass bit of every active dof; inactive dofs are never written.
__global__ void __launch_bounds__(kBlock) k_pstep_tape(Grid g, const int4* __restrict__ rt,
                                                       const int4* __restrict__ ct, const float* __restrict__ u,
                                                       float* __restrict__ P1, float* __restrict__ P2,
                                                       const float* __restrict__ Ph1, const float* __restrict__ Ph2,
                                                       float* __restrict__ Pb1, float* __restrict__ Pb2,
                                                       const Coef* __restrict__ ck, uint8_t* __restrict__ M1,
                                                       uint8_t* __restrict__ M2) {
  Pix q;
  if (!pixel_of(g, rt, ct, q)) return;
  const Coef c = *ck;
  const int W2 = g.W + g.NC;
  const size_t px = (size_t)q.i * g.W + q.j;
  const float uc = u[px];
  const size_t et = (size_t)(q.i + q.a) * g.W + q.j;
  if (q.i > q.r0) p_tape_dof(P1, Pb1, Ph1, M1, et, uc - u[px - g.W], c);
  else if (q.a > 0) p_tape_dof(P1, Pb1, Ph1, M1, et, uc, c);
  const size_t el = (size_t)q.i * W2 + q.j + q.b;
  if (q.j > q.c0) p_tape_dof(P2, Pb2, Ph2, M2, el, uc - u[px - 1], c);
  else if (q.b > 0) p_tape_dof(P2, Pb2, Ph2, M2, el, uc, c);
  if (q.i == q.r1 - 1 && q.a + 1 < g.NR) p_tape_dof(P1, Pb1, Ph1, M1, et + g.W, -uc, c);
  if (q.j == q.c1 - 1 && q.b + 1 < g.NC) p_tape_dof(P2, Pb2, Ph2, M2, el + 1, -uc, c);
}

// ---- reverse of one inner iteration

// Partial derivatives of u' = prox(ubar) (Section 3 proximity maps) at one pixel:
// dub = du'/dubar, df = du'/df, dal = du'/dalpha.  fv is f (L2, L1) or f itself for
// SEG (g is formed here); decisions use the forward's float arithmetic.
template <int FID>
__device__ __forceinline__ void prox_partials(float ub, float fv, bool in_d, float c1, float c2, const Coef& c,
                                              float& dub, float& df, float& dal) {
  if (FID == FID_SEG) {
    const float gv = (fv - c1) * (fv - c1) - (fv - c2) * (fv - c2);
    const float x = fmaf(-c.s, gv, ub);
    const bool pass = x >= 0.0f && x <= 1.0f;
    // x = ubar - sigma_k alpha g(f), g'(f) = 2 (c2 - c1)
    dub = pass ? 1.0f : 0.0f;
    dal = pass ? -c.sig * gv : 0.0f;
    df = pass ? -c.s * (2.0f * (c2 - c1)) : 0.0f;
    return;
  }
  if (in_d) {  // prox is the identity on the inpainting domain
    dub = 1.0f;
    df = 0.0f;
    dal = 0.0f;
    return;
  }
  if (FID == FID_L2) {
    // u' = (ubar + s f) / (1 + s), s = sigma_k alpha: du'/dalpha = sigma_k (f - ubar) / (1 + s)^2
    dub = c.ua;
    df = c.ub;
    dal = c.sig * c.ua * c.ua * (fv - ub);
    return;
  }
  // L1: u' = ubar - s sign(v) if |v| > s (v = ubar - f), else f
  const float v = ub - fv;
  const bool pass = fabsf(v) - c.s > 0.0f;
  dub = pass ? 1.0f : 0.0f;
  df = pass ? 0.0f : 1.0f;
  dal = pass ? (v > 0.0f ? -c.sig : c.sig) : 0.0f;
}

__device__ __forceinline__ float at_of(const uint8_t* __restrict__ M, const float* __restrict__ AP,
                                       const float* __restrict__ AQ, size_t e, float opq) {
  return M[e] ? AP[e] + opq * AQ[e] : 0.0f;
}

// Aal: one float64 partial sum of the alpha adjoint per block (block b of the 2-D grid
// always covers the same pixels, so the sums are deterministic).
template <int FID, bool MASK>
__global__ void __launch_bounds__(kBlock) k_adj_u(Grid g, const int4* __restrict__ rt, const int4* __restrict__ ct,
                                                  float c1, float c2, const float* __restrict__ f,
                                                  const uint8_t* __restrict__ mask, const float* __restrict__ ubar,
                                                  const uint8_t* __restrict__ M1, const uint8_t* __restrict__ M2,
                                                  const float* __restrict__ AP1, const float* __restrict__ AP2,
                                                  const float* __restrict__ AQ1, const float* __restrict__ AQ2,
                                                  float* __restrict__ Au, float* __restrict__ Ad,
                                                  float* __restrict__ Af, double* __restrict__ Aal,
                                                  const Coef* __restrict__ ck) {
  const Coef c = *ck;
  double acc = 0.0;
  Pix q;
  if (pixel_of(g, rt, ct, q)) {
    const float opq = 1.0f + c.th;
    const int W2 = g.W + g.NC;
    const size_t px = (size_t)q.i * g.W + q.j;
    const size_t et = (size_t)(q.i + q.a) * g.W + q.j, eb = et + g.W;
    const size_t el = (size_t)q.i * W2 + q.j + q.b, er = el + 1;
    const float dv = div_px(c.pc * at_of(M1, AP1, AQ1, et, opq), c.pc * at_of(M1, AP1, AQ1, eb, opq),
                            c.pc * at_of(M2, AP2, AQ2, el, opq), c.pc * at_of(M2, AP2, AQ2, er, opq));
    const float aun = Au[px] - dv;
    float dub, df, dal;
    prox_partials<FID>(ubar[px], f[px], MASK && mask[px], c1, c2, c, dub, df, dal);
    const float aub = dub * aun;
    Au[px] = aub;
    Ad[px] = c.sig * aub;
    if (df != 0.0f) Af[px] += df * aun;
    acc = (double)dal * (double)aun;
  }
  const int tid = threadIdx.y * kBX + threadIdx.x;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  __shared__ double sw[kBlock / 32];
  if ((tid & 31) == 0) sw[tid >> 5] = acc;
  __syncthreads();
  if (tid == 0) {
    double t = 0.0;
    for (int w = 0; w < kBlock / 32; ++w) t += sw[w];
    Aal[blockIdx.y * gridDim.x + blockIdx.x] += t;
  }
}

// AP, AQ, APhat of one dof.  first: APhat starts at 0 (first reverse step of an outer
// iteration); last: the adjoint of p~^n = p_0 = q_0 = (phat's copy) is folded into AP.
__device__ __forceinline__ void adj_dof(float* __restrict__ AP, float* __restrict__ AQ, float* __restrict__ APh,
                                        const uint8_t* __restrict__ M, size_t e, float aq_new, const Coef& c,
                                        float opq, bool first, bool last) {
  const float aq = AQ[e];
  const float at = M[e] ? AP[e] + opq * aq : 0.0f;
  const float aph = (first ? 0.0f : APh[e]) + c.pb * at;
  const float ap = c.pa * at - c.th * aq;
  APh[e] = aph;
  if (last) {
    AP[e] = (ap + aq_new) + aph;
    AQ[e] = 0.0f;
  } else {
    AP[e] = ap;
    AQ[e] = aq_new;
  }
}

__global__ void __launch_bounds__(kBlock) k_adj_p(Grid g, const int4* __restrict__ rt, const int4* __restrict__ ct,
                                                  const uint8_t* __restrict__ M1, const uint8_t* __restrict__ M2,
                                                  const float* __restrict__ Ad, float* __restrict__ AP1,
                                                  float* __restrict__ AP2, float* __restrict__ AQ1,
                                                  float* __restrict__ AQ2, float* __restrict__ APh1,
                                                  float* __restrict__ APh2, const Coef* __restrict__ ck, int first,
                                                  int last) {
  Pix q;
  if (!pixel_of(g, rt, ct, q)) return;
  const Coef c = *ck;
  const float opq = 1.0f + c.th;
  const bool fi = first != 0, la = last != 0;
  const int W2 = g.W + g.NC;
  const size_t px = (size_t)q.i * g.W + q.j;
  const float ad = Ad[px];
  const size_t et = (size_t)(q.i + q.a) * g.W + q.j;
  // d = div q: the dof between pixels m (above / left) and n of one tile enters
  // d_m with + and d_n with -, so AQ = Ad_m - Ad_n (a missing pixel counts 0)
  if (q.i > q.r0) adj_dof(AP1, AQ1, APh1, M1, et, Ad[px - g.W] - ad, c, opq, fi, la);
  else if (q.a > 0) adj_dof(AP1, AQ1, APh1, M1, et, -ad, c, opq, fi, la);
  const size_t el = (size_t)q.i * W2 + q.j + q.b;
  if (q.j > q.c0) adj_dof(AP2, AQ2, APh2, M2, el, Ad[px - 1] - ad, c, opq, fi, la);
  else if (q.b > 0) adj_dof(AP2, AQ2, APh2, M2, el, -ad, c, opq, fi, la);
  if (q.i == q.r1 - 1 && q.a + 1 < g.NR) adj_dof(AP1, AQ1, APh1, M1, et + g.W, ad, c, opq, fi, la);
  if (q.j == q.c1 - 1 && q.b + 1 < g.NC) adj_dof(AP2, AQ2, APh2, M2, el + 1, ad, c, opq, fi, la);
}

// ---- reverse of the interface step of outer iteration n
//   lambda^{n+1} = lambda^n + sigma B (2 p~^n - p~^{n-1}),  phat = p~^n - tau B^* lambda^{n+1}
// With AL the adjoint of lambda^{n+1} carried from iteration n+1 and APp the adjoint
// of p~^n's interface values through iteration n+1's extrapolation:
//   AL'  = AL - tau B APhat
//   AP  += APp + 2 sigma B^* AL'      (on the interface sides; AP already holds the
//                                      local solve's and phat's contributions)
//   AL  <- AL' (adjoint of lambda^n),  APp <- -sigma B^* AL' (adjoint of p~^{n-1})
__global__ void k_adj_interface(Grid g, float sigma, float tau, float* __restrict__ AP1, float* __restrict__ AP2,
                                const float* __restrict__ APh1, const float* __restrict__ APh2,
                                float* __restrict__ ALh, float* __restrict__ ALv, Strips APp) {
  const int nh = (g.NR - 1) * g.W, nv = (g.NC - 1) * g.H;
  const int W2 = g.W + g.NC;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < nh + nv; e += gridDim.x * blockDim.x) {
    if (e < nh) {
      const int a = e / g.W, j = e % g.W;
      const int rs = part_start(a + 1, g.H, g.NR) + a;
      const size_t s = (size_t)rs * g.W + j, t = s + g.W;
      const float al = ALh[e] - tau * (APh1[s] - APh1[t]);
      AP1[s] += APp.SB[e] + 2.0f * sigma * al;
      AP1[t] += APp.ST[e] - 2.0f * sigma * al;
      ALh[e] = al;
      APp.SB[e] = -sigma * al;
      APp.ST[e] = sigma * al;
    } else {
      const int q = e - nh, b = q / g.H, i = q % g.H;
      const int cs = part_start(b + 1, g.W, g.NC) + b;
      const size_t s = (size_t)i * W2 + cs, t = s + 1;
      const float al = ALv[q] - tau * (APh2[s] - APh2[t]);
      AP2[s] += APp.SR[q] + 2.0f * sigma * al;
      AP2[t] += APp.SL[q] - 2.0f * sigma * al;
      ALv[q] = al;
      APp.SR[q] = -sigma * al;
      APp.SL[q] = sigma * al;
    }
  }
}

// Af += du^0/df Au (u^0 = f off the inpainting domain for L2/L1; constant otherwise)
__global__ void k_adj_initial(long long n, int fid, const uint8_t* __restrict__ mask, const float* __restrict__ Au,
                              float* __restrict__ Af) {
  if (fid == FID_SEG) return;
  for (long long px = blockIdx.x * (long long)blockDim.x + threadIdx.x; px < n;
       px += (long long)gridDim.x * blockDim.x)
    if (!(mask && mask[px])) Af[px] += Au[px];
}

// Sum of n doubles: per-thread sums, warp shuffles, block partials, and the last block
// to finish adds the partials in block order (deterministic).
constexpr int kSumBlocks = 152 * 4;

__global__ void __launch_bounds__(kBlock) k_sum_f64(const double* __restrict__ x, long long n,
                                                    double* __restrict__ partials, unsigned int* __restrict__ counter,
                                                    double* __restrict__ out) {
  double v = 0.0;
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n; q += (long long)gridDim.x * blockDim.x)
    v += x[q];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  __shared__ double sw[kBlock / 32];
  __shared__ bool last;
  if ((threadIdx.x & 31) == 0) sw[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double bsum = 0.0;
    for (int w = 0; w < kBlock / 32; ++w) bsum += sw[w];
    partials[blockIdx.x] = bsum;
    __threadfence();
    last = atomicAdd(counter, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (last && threadIdx.x == 0) {
    __threadfence();
    double t = 0.0;
    for (int q = 0; q < (int)gridDim.x; ++q) t += ((volatile double*)partials)[q];
    out[0] = t;
    *counter = 0u;
  }
}

}  // namespace

cudaError_t launch_ustep_tape(const LocalArgs& a, const int4* rt, const int4* ct, const float* Pb1, const float* Pb2,
                              const Coef* ck, int fid, float* ubar_out, cudaStream_t st) {
  const Grid& g = a.g;
  const dim3 grid = pixel_grid(g), block(kBX, kBY);
  const bool m = a.mask != nullptr;
#define USTEP(F, MK) \
  k_ustep_tape<F, MK><<<grid, block, 0, st>>>(g, rt, ct, a.c1, a.c2, a.f, a.mask, a.u, Pb1, Pb2, ck, ubar_out)
  if (fid == FID_L2) {
    if (m) USTEP(FID_L2, true); else USTEP(FID_L2, false);
  } else if (fid == FID_L1) {
    if (m) USTEP(FID_L1, true); else USTEP(FID_L1, false);
  } else {
    USTEP(FID_SEG, false);
  }
#undef USTEP
  return cudaGetLastError();
}

cudaError_t launch_pstep_tape(const LocalArgs& a, const int4* rt, const int4* ct, const float* Ph1, const float* Ph2,
                              float* Pb1, float* Pb2, const Coef* ck, uint8_t* M1, uint8_t* M2, cudaStream_t st) {
  const Grid& g = a.g;
  k_pstep_tape<<<pixel_grid(g), dim3(kBX, kBY), 0, st>>>(g, rt, ct, a.u, a.P1, a.P2, Ph1, Ph2, Pb1, Pb2, ck, M1,
                                                          M2);
  return cudaGetLastError();
}

cudaError_t launch_adj_inner(const AdjArgs& r, const Coef* ck, const float* ubar, const uint8_t* M1,
                             const uint8_t* M2, bool first, bool last, cudaStream_t st) {
  const Grid& g = r.g;
  const dim3 grid = pixel_grid(g), block(kBX, kBY);
  const bool m = r.mask != nullptr;
#define ADJ_U(F, MK)                                                                                           \
  k_adj_u<F, MK><<<grid, block, 0, st>>>(g, r.rowtab, r.coltab, r.c1, r.c2, r.f, r.mask, ubar, M1, M2, r.AP1, \
                                         r.AP2, r.AQ1, r.AQ2, r.Au, r.Ad, r.Af, r.Aal, ck)
  if (r.fid == FID_L2) {
    if (m) ADJ_U(FID_L2, true); else ADJ_U(FID_L2, false);
  } else if (r.fid == FID_L1) {
    if (m) ADJ_U(FID_L1, true); else ADJ_U(FID_L1, false);
  } else {
    ADJ_U(FID_SEG, false);
  }
#undef ADJ_U
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_adj_p<<<grid, block, 0, st>>>(g, r.rowtab, r.coltab, M1, M2, r.Ad, r.AP1, r.AP2, r.AQ1, r.AQ2, r.APh1, r.APh2,
                                  ck, first ? 1 : 0, last ? 1 : 0);
  return cudaGetLastError();
}

cudaError_t launch_adj_interface(const AdjArgs& r, float sigma, float tau, cudaStream_t st) {
  const Grid& g = r.g;
  const int n = (g.NR - 1) * g.W + (g.NC - 1) * g.H;
  if (n == 0) return cudaSuccess;
  k_adj_interface<<<nblocks(n), kBlock, 0, st>>>(g, sigma, tau, r.AP1, r.AP2, r.APh1, r.APh2, r.ALh, r.ALv, r.APp);
  return cudaGetLastError();
}

cudaError_t launch_adj_initial(const AdjArgs& r, cudaStream_t st) {
  const long long n = (long long)r.g.H * r.g.W;
  k_adj_initial<<<nblocks(n), kBlock, 0, st>>>(n, r.fid, r.mask, r.Au, r.Af);
  return cudaGetLastError();
}

int sum_f64_partials_count() { return kSumBlocks; }

long long adj_alpha_slots(const Grid& g) {
  const dim3 d = pixel_grid(g);
  return (long long)d.x * d.y;
}

cudaError_t launch_sum_f64(const double* x, long long n, double* partials, unsigned int* counter, double* out,
                           cudaStream_t st) {
  k_sum_f64<<<kSumBlocks, kBlock, 0, st>>>(x, n, partials, counter, out);
  return cudaGetLastError();
}

}  // namespace ddtv
