// Pointwise arithmetic of one local primal-dual iteration (Section 5, local
// solver: the accelerated primal-dual algorithm with the dual field p as the
// uniformly convex variable).  Every kernel that runs an inner iteration (fused and
// plain paths, full-dimension comparator) uses these functions, so the paths agree
// bit for bit.  Compiled with --fmad=false: only the fmaf calls written here fuse.
#pragma once

#include <cstdint>

namespace ddtv {

enum { FID_L2 = 0, FID_L1 = 1, FID_SEG = 2 };

// Coefficients of inner iteration k, computed on the host in double precision:
//   sig = sigma_k                       u-step size
//   ua  = 1 / (1 + sigma_k alpha)       L2 prox: u = ua * ubar + ub * f
//   ub  = sigma_k alpha / (1 + sigma_k alpha)
//   s   = sigma_k alpha                 L1 shrink threshold, SEG step on g
//   pa  = tau / (tau + tau_k)           prox of G^*: p = proj_C(pa p + pc Du + pb phat)
//   pc  = tau tau_k / (tau + tau_k)
//   pb  = tau_k / (tau + tau_k)
//   th  = theta_k = 1 / sqrt(1 + 2 gamma tau_k)   extrapolation pbar = pn + th (pn - p)
struct Coef {
  float sig, ua, ub, s, pa, pc, pb, th;
};

// div_s p at a pixel from the normal components on its four sides
// (outflow: bottom - top + right - left, Section 2.3)
__device__ __forceinline__ float div_px(float top, float bot, float left, float right) {
  return ((bot - top) + right) - left;
}

// u <- prox_{sigma_k alpha F}(u + sigma_k div pbar) (Section 3 proximity maps).
// fg is f (L2, L1) or g = (f - c1)^2 - (f - c2)^2 (SEG); in_d marks the inpainting
// domain D, where the L2/L1 fidelity vanishes and the prox is the identity.
template <int FID>
__device__ __forceinline__ float prox_ubar(float ubar, float fg, bool in_d, const Coef& c);

template <int FID>
__device__ __forceinline__ float u_update(float u, float d, float fg, bool in_d, const Coef& c) {
  return prox_ubar<FID>(fmaf(c.sig, d, u), fg, in_d, c);
}

// Projection onto [-lim, lim] (lim >= 0), the pointwise constraint set of the dual
// field (|p| <= 1 on an edge, 0 on an edge of the image boundary): one min.xorsign.abs,
// whose magnitude is min(|x|, lim) and whose sign is sign(x) xor sign(lim) = sign(x);
// the value of fminf(fmaxf(x, -lim), lim) for every x that is not NaN.
__device__ __forceinline__ float clamp_abs(float x, float lim) {
  float r;
  asm("min.xorsign.abs.f32 %0, %1, %2;" : "=f"(r) : "f"(x), "f"(lim));
  return r;
}

// prox_{sigma_k alpha F} at ubar = u + sigma_k div pbar
template <int FID>
__device__ __forceinline__ float prox_ubar(float ubar, float fg, bool in_d, const Coef& c) {
  if (FID == FID_SEG) {
    const float x = fmaf(-c.s, fg, ubar);
    return fminf(fmaxf(x, 0.0f), 1.0f);
  }
  if (in_d) return ubar;
  if (FID == FID_L2) return fmaf(c.ub, fg, c.ua * ubar);
  // L1: f + shr(ubar - f, s) with shr(v, s) = max(|v| - s, 0) sign(v), evaluated as
  // ubar - P_[-s,s](ubar - f) (the same map: v - P(v) = shr(v, s)), one projection
  const float v = ubar - fg;
  return ubar - clamp_abs(v, c.s);
}

// Argument of the projection in the p-step: (tau (p + tau_k Du) + tau_k phat) / (tau + tau_k).
__device__ __forceinline__ float p_target(float p, float du, float phat, const Coef& c) {
  return fmaf(c.pc, du, fmaf(c.pa, p, c.pb * phat));
}

// One dof of the p-step: q = p + tau_k Du, p_new = proj_[-1,1]((tau q + tau_k phat) /
// (tau + tau_k)), pbar = p_new + theta_k (p_new - p).
__device__ __forceinline__ void p_update(float& p, float& pbar, float du, float phat, const Coef& c) {
  const float t = p_target(p, du, phat, c);
  const float pn = clamp_abs(t, 1.0f);
  pbar = fmaf(c.th, pn - p, pn);
  p = pn;
}

// proximal centre phat = p~^n - tau B^* lambda on an interface side (Algorithm 1):
// the s-side (bottom/right) copy gets -tau lambda, the t-side (top/left) copy +tau lambda
__device__ __forceinline__ float phat_s(float p, float lam, float tau) { return fmaf(-tau, lam, p); }
__device__ __forceinline__ float phat_t(float p, float lam, float tau) { return fmaf(tau, lam, p); }

// first pixel row (column) of tile a when len pixels are split into n tiles
__host__ __device__ __forceinline__ int part_start(int a, int len, int n) {
  return (int)(((long long)a * len) / n);
}

// the tile that pixel row (column) i belongs to
__host__ __device__ __forceinline__ int part_of(int i, int len, int n) {
  return (int)(((long long)(i + 1) * n - 1) / len);
}

}  // namespace ddtv
