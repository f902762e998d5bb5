// Fused local solver: all inner iterations of one outer iteration of Algorithm 1 for
// every subdomain in one launch (Section 5, local problem eq. local, solved by the
// accelerated primal-dual algorithm with the dual field p as the uniformly convex
// variable; the projection onto the box C of eq. proj_C is fused into the p-step).
//
// Mapping.  One subdomain (tile of mr x mc pixels, mc <= BW, mr <= CL*TR*R) is owned
// by a thread-block cluster of CL CTAs; CTA `rank` owns a band of TR*R tile rows and
// thread (x, y) of it owns pixel column x and the R consecutive band rows y*R ..
// y*R+R-1 (the 32 lanes of a warp are 32 adjacent columns).  Registers hold, per
// pixel: u, the torn dual dofs p1 (top edge) and p2 (left edge), their proximal
// centres h1, h2 and the extrapolation pbar1.  Shared memory holds what neighbours
// read: u (zero-padded on the left), pbar2 (the tile's right side in column mc),
// f (or g), the first-row pbar1 of every thread row, and two halo rows that the
// neighbouring CTAs of the cluster write through distributed shared memory (u of
// the row above the band, pbar1 of the row below it).  The halo of the tile's top
// row and the padding left of column 0 stay zero, so the interface formulas
// D_s u = +u on the top and left sides need no branch; an inactive side (image
// boundary) is kept at 0 by clamping its dofs to [-0, 0].
//
// Synchronisation per inner iteration: two CTA barriers and two phases of the
// cluster barrier.  In each half-step a CTA first computes the row its neighbour
// needs, stores it into the neighbour's halo, arrives on the cluster barrier, then
// computes its other rows; the matching wait comes a half-step later, so the
// cross-SM latency of the cluster barrier hides behind the interior work.  Only
// warps that wrote to a neighbour arrive with release semantics.
#include "internal.cuh"
#include "fused_common.cuh"

namespace ddtv {

namespace {

template <int BW, int R, int TR>
struct SmemLayout {
  static constexpr int BAND = TR * R;
  static constexpr int US = BW + 1;                    // row stride of u (index 0 = zero pad)
  static constexpr int QS = BW + 1;                    // row stride of pbar2 (index mc = right side)
  static constexpr int U = 0;                          // BAND x US   u of the band
  static constexpr int UH = U + BAND * US;             // US          u of the row above the band
  static constexpr int Q2 = UH + US;                   // BAND x QS   pbar2
  static constexpr int Q1 = Q2 + BAND * QS;            // TR x BW     pbar1 of each thread row's first row
  static constexpr int Q1H = Q1 + TR * BW;             // BW          pbar1 of the row below the band
  static constexpr int F = Q1H + BW;                   // BAND x BW   f (or g)
  static constexpr int PR = F + BAND * BW;             // BAND        right-side p
  static constexpr int HR = PR + BAND;                 // BAND        right-side phat
  static constexpr int FLOATS = HR + BAND;
  static constexpr size_t BYTES = sizeof(float) * FLOATS;
};

// ADAPT: adaptive inner stopping (Section 5, eq. stop_inner1).  Every thread sums
// (p^{k+1} - p^k)^2 and (p^{k+1})^2 over the tile dofs it owns, each warp adds its
// threads' sums (float32, fixed shuffle order), one thread adds the warps' sums in
// float64 in a fixed order and stores the CTA's pair into every cluster CTA's slot
// array through DSMEM, and after one more cluster barrier phase one thread of every
// CTA adds the CL pairs in rank order and shares the decision through shared memory:
// all CTAs of the tile take the same decision.  (Float64 work stays with one thread:
// the float64 pipe of this GPU is narrow.)  The u-step's first cluster wait is then
// taken at the end of the previous iteration's p-step instead.
template <int BW, int R, int TR, int CL, int FID, bool MASK, bool ADAPT>
__global__ void __launch_bounds__(BW* TR, (BW * TR <= 256 ? 2 : 1)) k_fused(const LocalArgs A) {
  using L = SmemLayout<BW, R, TR>;
  constexpr int BAND = L::BAND;
  extern __shared__ float smem[];
  __shared__ double sRed[2 * CL];            // adaptive stop: per-rank (sum dp^2, sum p^2)
  __shared__ double sWarp[2 * (BW * TR / 32)];
  __shared__ int sStop;                      // adaptive stop: the CTA's decision
  float* sU = smem + L::U;
  float* sUh = smem + L::UH;
  float* sQ2 = smem + L::Q2;
  float* sQ1 = smem + L::Q1;
  float* sQ1h = smem + L::Q1H;
  float* sF = smem + L::F;
  float* sPR = smem + L::PR;
  float* sHR = smem + L::HR;

  const Grid g = A.g;
  const int rank = CL > 1 ? (int)blockIdx.x : 0;
  const int b = blockIdx.y, a = blockIdx.z;
  const int r0 = part_start(a, g.H, g.NR), mr = part_start(a + 1, g.H, g.NR) - r0;
  const int c0 = part_start(b, g.W, g.NC), mc = part_start(b + 1, g.W, g.NC) - c0;
  const bool s_top = a > 0, s_bot = a + 1 < g.NR, s_lft = b > 0, s_rgt = b + 1 < g.NC;
  const int j = threadIdx.x, ty = threadIdx.y;
  const int lr0 = ty * R;            // first band row of this thread
  const int i0 = rank * BAND + lr0;  // first tile row of this thread
  const bool col_ok = j < mc;
  const int W2 = g.W + g.NC;
  const int gj = c0 + j;
  const float tau = A.tau;
  // clamp limits: 0 keeps an image-boundary dof at 0
  const float lim_left = (j == 0 && !s_lft) ? 0.f : 1.f;
  const float lim_top = (i0 == 0 && !s_top) ? 0.f : 1.f;  // applies to r = 0 only
  const int rb = mr - 1 - i0;                              // r of the tile's last row, if in [0, R)
  // the band's last row is read by the CTA below, its first row by the CTA above
  const bool push_down = CL > 1 && ty == TR - 1 && rank + 1 < CL;
  const bool push_up = CL > 1 && ty == 0 && rank > 0;
  uint32_t remote_uh = 0, remote_q1h = 0;
  if (CL > 1) {
    if (push_down) remote_uh = map_rank(smem_addr(sUh + 1 + j), rank + 1);
    if (push_up) remote_q1h = map_rank(smem_addr(sQ1h + j), rank - 1);
  }

  float u[R], p1[R], p2[R], h1[R], h2[R], q1[R];
  uint32_t in_d = 0;
  float pB = 0.f, hB = 0.f, qB = 0.f;  // bottom side of the tile (thread row holding row mr-1)

  // ---- load the tile's state and build the proximal centre
  // The tile's first row sees u = 0 above it.  The other CTAs' halos are written by
  // their neighbours before every read; sQ1h is only read by rows that either have a
  // neighbour below or lie outside the tile (their values are never stored).
  if (rank == 0) {
    if (j == 0) sUh[0] = 0.f;
    sUh[1 + j] = 0.f;
  }
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const int i = i0 + r;
    float uv = 0.f, fv = 0.f, a1 = 0.f, a2 = 0.f, b1 = 0.f, b2 = 0.f;
    if (col_ok && i < mr) {
      const int gi = r0 + i;
      const size_t px = (size_t)gi * g.W + gj;
      uv = A.u[px];
      fv = A.f[px];
      if (FID == FID_SEG) fv = (fv - A.c1) * (fv - A.c1) - (fv - A.c2) * (fv - A.c2);
      if (MASK && A.mask[px]) in_d |= 1u << r;
      a1 = A.P1[(size_t)(gi + a) * g.W + gj];
      a2 = A.P2[(size_t)gi * W2 + gj + b];
      b1 = (i == 0 && s_top) ? phat_t(a1, A.lamh[(size_t)(a - 1) * g.W + gj], tau) : a1;
      b2 = (j == 0 && s_lft) ? phat_t(a2, A.lamv[(size_t)(b - 1) * g.H + gi], tau) : a2;
      if (i == mr - 1 && s_bot) {
        pB = A.P1[(size_t)(gi + a + 1) * g.W + gj];
        hB = phat_s(pB, A.lamh[(size_t)a * g.W + gj], tau);
      }
      if (j == mc - 1) {
        float pr = 0.f, hr = 0.f;
        if (s_rgt) {
          pr = A.P2[(size_t)gi * W2 + gj + b + 1];
          hr = phat_s(pr, A.lamv[(size_t)b * g.H + gi], tau);
        }
        sPR[lr0 + r] = pr;
        sHR[lr0 + r] = hr;
        sQ2[(lr0 + r) * L::QS + mc] = pr;
      }
    }
    u[r] = uv;
    p1[r] = a1;
    p2[r] = a2;
    h1[r] = b1;
    h2[r] = b2;
    q1[r] = a1;
    sF[(lr0 + r) * BW + j] = fv;
    sU[(lr0 + r) * L::US] = 0.f;  // left padding (every thread writes the same value)
    if (col_ok) sQ2[(lr0 + r) * L::QS + j] = a2;
  }
  qB = pB;
  sQ1[ty * BW + j] = q1[0];
  if (push_up) st_cluster(remote_q1h, q1[0]);
  __syncthreads();
  if (CL > 1) {
    if (push_up) cluster_arrive<true>(); else cluster_arrive<false>();
  }

  const float4* coef4 = reinterpret_cast<const float4*>(A.coef);

  auto u_px = [&](int r, const Coef& c) {
    const int lr = lr0 + r;
    float below;
    if (r == rb) below = qB;                                 // the tile's bottom side
    else if (r + 1 < R) below = q1[r + 1];
    else if (ty + 1 < TR) below = sQ1[(ty + 1) * BW + j];
    else below = sQ1h[j];                                    // first row of the band below
    const float left = sQ2[lr * L::QS + j];
    const float right = sQ2[lr * L::QS + j + 1];
    const float d = div_px(q1[r], below, left, right);
    u[r] = u_update<FID>(u[r], d, sF[lr * BW + j], MASK && ((in_d >> r) & 1u), c);
    sU[lr * L::US + j + 1] = u[r];
  };

  float sd = 0.f, sp = 0.f;  // adaptive stop: this thread's sums over its tile dofs
  auto res_add = [&](float po, float pn) {
    const float dp = pn - po;
    sd = fmaf(dp, dp, sd);
    sp = fmaf(pn, pn, sp);
  };

  auto p_px = [&](int r, const Coef& c) {
    const int lr = lr0 + r;
    const bool in_tile = ADAPT && col_ok && i0 + r < mr;
    float above;
    if (r > 0) above = u[r - 1];
    else if (ty > 0) above = sU[(lr - 1) * L::US + j + 1];
    else above = sUh[j + 1];                                 // 0 above the tile's first row
    const float o1 = p1[r], o2 = p2[r];
    p_update_lim(p1[r], q1[r], u[r] - above, h1[r], c, r == 0 ? lim_top : 1.f);
    float q2;
    p_update_lim(p2[r], q2, u[r] - sU[lr * L::US + j], h2[r], c, lim_left);
    if (in_tile) {
      res_add(o1, p1[r]);
      res_add(o2, p2[r]);
    }
    if (r == rb && s_bot) {
      const float oB = pB;
      p_update(pB, qB, -u[r], hB, c);
      if (in_tile) res_add(oB, pB);
    }
    if (j == mc - 1 && s_rgt) {
      float pr = sPR[lr], qr;
      const float orr = pr;
      p_update(pr, qr, -u[r], sHR[lr], c);
      if (in_tile) res_add(orr, pr);
      sPR[lr] = pr;
      sQ2[lr * L::QS + mc] = qr;
    }
    if (col_ok) sQ2[lr * L::QS + j] = q2;
  };

  // ---- inner iterations
  int k_run = A.K;
  for (int k = 0; k < A.K; ++k) {
    const float4 ca = __ldg(coef4 + 2 * k), cb = __ldg(coef4 + 2 * k + 1);
    const Coef c{ca.x, ca.y, ca.z, ca.w, cb.x, cb.y, cb.z, cb.w};
    // u-step: the band's last row first (the CTA below needs it)
    if (CL > 1 && (!ADAPT || k == 0)) cluster_wait();
    u_px(R - 1, c);
    if (push_down) st_cluster(remote_uh, u[R - 1]);
    if (CL > 1) {
      if (push_down) cluster_arrive<true>(); else cluster_arrive<false>();
    }
#pragma unroll
    for (int r = 0; r + 1 < R; ++r) u_px(r, c);
    __syncthreads();
    // p-step: the band's first row first (the CTA above needs its pbar1)
    if (CL > 1) cluster_wait();
    p_px(0, c);
    sQ1[ty * BW + j] = q1[0];
    if (push_up) st_cluster(remote_q1h, q1[0]);
    if (CL > 1) {
      if (push_up) cluster_arrive<true>(); else cluster_arrive<false>();
    }
#pragma unroll
    for (int r = 1; r < R; ++r) p_px(r, c);
    __syncthreads();
    if (ADAPT) {
      // warp sums in float32 (fixed shuffle order), then one thread adds the warps' sums in
      // order in float64
      const int tid = ty * BW + j, lane = tid & 31, wid = tid >> 5;
      float wd = sd, wp = sp;
      sd = sp = 0.f;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        wd += __shfl_down_sync(0xffffffffu, wd, o);
        wp += __shfl_down_sync(0xffffffffu, wp, o);
      }
      if (lane == 0) {
        sWarp[2 * wid] = wd;
        sWarp[2 * wid + 1] = wp;
      }
      __syncthreads();
      if (CL > 1) cluster_wait();  // the p-step's cluster phase (halo rows of pbar1)
      if (tid == 0) {
        double td = 0.0, tp = 0.0;
        for (int w = 0; w < BW * TR / 32; ++w) {
          td += sWarp[2 * w];
          tp += sWarp[2 * w + 1];
        }
        if (CL > 1) {
          for (int q = 0; q < CL; ++q) {
            st_cluster_f64(map_rank(smem_addr(sRed + 2 * rank), q), td);
            st_cluster_f64(map_rank(smem_addr(sRed + 2 * rank + 1), q), tp);
          }
        } else {
          sRed[0] = td;
          sRed[1] = tp;
        }
      }
      if (CL > 1) {
        cluster_arrive<true>();
        cluster_wait();
      } else {
        __syncthreads();
      }
      if (tid == 0) {
        double td = 0.0, tp = 0.0;
        for (int q = 0; q < CL; ++q) {
          td += sRed[2 * q];
          tp += sRed[2 * q + 1];
        }
        sStop = (tp == 0.0 || td < A.inner_tol2 * tp) ? 1 : 0;
      }
      __syncthreads();
      if (sStop) {
        k_run = k + 1;
        break;
      }
    }
  }
  if (CL > 1 && !ADAPT) cluster_wait();  // no CTA leaves while a neighbour may still write its halo
  if (ADAPT && rank == 0 && j == 0 && ty == 0) {
    A.inner_used[a * g.NC + b] = k_run;
    atomicMax(A.inner_max, k_run);
    atomicAdd(A.inner_work, (unsigned long long)mr * (unsigned long long)mc * (unsigned long long)k_run);
  }

  // ---- store u^{n+1}, p~^{n+1} and the interface strips
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const int i = i0 + r;
    if (col_ok && i < mr) {
      const int gi = r0 + i;
      A.u[(size_t)gi * g.W + gj] = u[r];
      A.P1[(size_t)(gi + a) * g.W + gj] = p1[r];
      A.P2[(size_t)gi * W2 + gj + b] = p2[r];
      if (i == 0 && s_top) A.out.ST[(size_t)(a - 1) * g.W + gj] = p1[r];
      if (j == 0 && s_lft) A.out.SL[(size_t)(b - 1) * g.H + gi] = p2[r];
      if (i == mr - 1 && s_bot) {
        A.P1[(size_t)(gi + a + 1) * g.W + gj] = pB;
        A.out.SB[(size_t)a * g.W + gj] = pB;
      }
      if (j == mc - 1 && s_rgt) {
        const float pr = sPR[lr0 + r];
        A.P2[(size_t)gi * W2 + gj + b + 1] = pr;
        A.out.SR[(size_t)b * g.H + gi] = pr;
      }
    }
  }
}


template <int R, int TR, int CL, int MINB, int FID, bool MASK>
__global__ void __launch_bounds__(128 * TR, MINB) k_fused_full(const LocalArgs A) {
  using L = FullLayout<R, TR>;
  constexpr int BW = L::BW, BAND = L::BAND;
  static_assert(CL * BAND == 128, "a cluster covers the 128 rows of a tile");
  extern __shared__ float smem[];
  float* sU = smem + L::U;
  float* sQ2 = smem + L::Q2;
  float* sQ1 = smem + L::Q1;
  float* sF = smem + L::F;
  float* sPR = smem + L::PR;
  float* sHR = smem + L::HR;
  float* sCo = smem + L::CO;

  const Grid g = A.g;
  const int rank = CL > 1 ? (int)blockIdx.x : 0;
  const int b = blockIdx.y, a = blockIdx.z;
  const int r0 = a * 128, c0 = b * 128;
  const bool s_top = a > 0, s_bot = a + 1 < g.NR, s_lft = b > 0, s_rgt = b + 1 < g.NC;
  const int j = threadIdx.x, ty = threadIdx.y;
  const int lr0 = ty * R;
  const int i0 = rank * BAND + lr0;
  const int W2 = g.W + g.NC;
  const int gj = c0 + j;
  const float tau = A.tau;
  const float lim_left = (j == 0 && !s_lft) ? 0.f : 1.f;
  const float lim_top = (i0 == 0 && !s_top) ? 0.f : 1.f;
  const bool last_row_here = rank == CL - 1 && ty == TR - 1;  // holds the tile's bottom row
  const bool push_down = CL > 1 && ty == TR - 1 && rank + 1 < CL;
  const bool push_up = CL > 1 && ty == 0 && rank > 0;
  // right side: lane l < R of warp 0 of each thread row owns the dof of band row lr0 + l
  const bool right_lane = s_rgt && j < R;
  uint32_t remote_u = 0, remote_q1 = 0;
  if (push_down) remote_u = map_rank(smem_addr(sU + 1 + j), rank + 1);           // row 0 (above) of rank + 1
  if (push_up) remote_q1 = map_rank(smem_addr(sQ1 + TR * BW + j), rank - 1);      // row TR (below) of rank - 1

  float u[R], p1[R], p2[R], h1[R], h2[R], q1[R];
  uint32_t in_d = 0;
  float pB = 0.f, hB = 0.f;

  for (int q = threadIdx.x + threadIdx.y * BW; q < 8 * min(A.K, L::kMaxSmemCoef); q += BW * TR)
    sCo[q] = reinterpret_cast<const float*>(A.coef)[q];
  if (rank == 0) sU[1 + j] = 0.f;  // u = 0 above the tile's first row
  if (j == 0) sU[0] = 0.f;
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const int gi = r0 + i0 + r;
    const size_t px = (size_t)gi * g.W + gj;
    u[r] = A.u[px];
    float fv = A.f[px];
    if (FID == FID_SEG) fv = (fv - A.c1) * (fv - A.c1) - (fv - A.c2) * (fv - A.c2);
    sF[(lr0 + r) * BW + j] = fv;
    if (MASK && A.mask[px]) in_d |= 1u << r;
    p1[r] = A.P1[(size_t)(gi + a) * g.W + gj];
    p2[r] = A.P2[(size_t)gi * W2 + gj + b];
    h1[r] = p1[r];
    h2[r] = p2[r];
    q1[r] = p1[r];
    sQ2[(lr0 + r) * L::QS + j] = p2[r];
    sU[(lr0 + r + 1) * L::US] = 0.f;
  }
  if (i0 == 0 && s_top) h1[0] = phat_t(p1[0], A.lamh[(size_t)(a - 1) * g.W + gj], tau);
  if (j == 0 && s_lft) {
#pragma unroll
    for (int r = 0; r < R; ++r) h2[r] = phat_t(p2[r], A.lamv[(size_t)(b - 1) * g.H + r0 + i0 + r], tau);
  }
  if (last_row_here) {
    if (s_bot) {
      pB = A.P1[(size_t)(r0 + 128 + a) * g.W + gj];
      hB = phat_s(pB, A.lamh[(size_t)a * g.W + gj], tau);
    }
    sQ1[TR * BW + j] = pB;
  }
  if (j < R) {  // right side of band row lr0 + j
    float pr = 0.f, hr = 0.f;
    if (s_rgt) {
      const int gi = r0 + i0 + j;
      pr = A.P2[(size_t)gi * W2 + c0 + 128 + b];
      hr = phat_s(pr, A.lamv[(size_t)b * g.H + gi], tau);
    }
    sPR[lr0 + j] = pr;
    sHR[lr0 + j] = hr;
    sQ2[(lr0 + j) * L::QS + 128] = pr;
  }
  sQ1[ty * BW + j] = q1[0];
  if (push_up) st_cluster(remote_q1, q1[0]);
  __syncthreads();
  if (CL > 1) {
    if (push_up) cluster_arrive<true>(); else cluster_arrive<false>();
  }

  float* sUr = sU + (lr0 + 1) * L::US + j + 1;  // u of band row lr0 + r, column j at sUr[r * US]
  float* sQ2r = sQ2 + lr0 * L::QS + j;
  const float* sFr = sF + lr0 * BW + j;

  for (int k = 0; k < A.K; ++k) {
    Coef c;
    if (k < L::kMaxSmemCoef) {
      const float4 ca = *reinterpret_cast<const float4*>(sCo + 8 * k);
      const float4 cb = *reinterpret_cast<const float4*>(sCo + 8 * k + 4);
      c = Coef{ca.x, ca.y, ca.z, ca.w, cb.x, cb.y, cb.z, cb.w};
    } else {
      c = A.coef[k];
    }
    // ---- u-step; the band's last row first
    if (CL > 1) cluster_wait();
#pragma unroll
    for (int rr = 0; rr < R; ++rr) {
      const int r = (rr + R - 1) % R;  // R-1, 0, 1, ..., R-2
      const float below = r + 1 < R ? q1[r + 1] : sQ1[(ty + 1) * BW + j];
      const float d = div_px(q1[r], below, sQ2r[r * L::QS], sQ2r[r * L::QS + 1]);
      u[r] = u_update<FID>(u[r], d, sFr[r * BW], MASK && ((in_d >> r) & 1u), c);
      sUr[r * L::US] = u[r];
      if (rr == 0) {
        if (push_down) st_cluster(remote_u, u[R - 1]);
        if (CL > 1) {
          if (push_down) cluster_arrive<true>(); else cluster_arrive<false>();
        }
      }
    }
    __syncthreads();
    // ---- p-step; the band's first row first
    if (CL > 1) cluster_wait();
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const float above = r > 0 ? u[r - 1] : sUr[-L::US];
      p_update_lim(p1[r], q1[r], u[r] - above, h1[r], c, r == 0 ? lim_top : 1.f);
      float q2;
      p_update_lim(p2[r], q2, u[r] - sUr[r * L::US - 1], h2[r], c, lim_left);
      sQ2r[r * L::QS] = q2;
      if (r == 0) {
        sQ1[ty * BW + j] = q1[0];
        if (push_up) st_cluster(remote_q1, q1[0]);
        if (CL > 1) {
          if (push_up) cluster_arrive<true>(); else cluster_arrive<false>();
        }
      }
    }
    if (last_row_here && s_bot) {  // the tile's bottom side: D_s u = -u
      float qB;
      p_update(pB, qB, -u[R - 1], hB, c);
      sQ1[TR * BW + j] = qB;
    }
    if (right_lane) {  // the tile's right side of band row lr0 + j: D_s u = -u
      const int lr = lr0 + j;
      float pr = sPR[lr], qr;
      p_update(pr, qr, -sU[(lr + 1) * L::US + 128], sHR[lr], c);
      sPR[lr] = pr;
      sQ2[lr * L::QS + 128] = qr;
    }
    __syncthreads();
  }
  if (CL > 1) cluster_wait();

#pragma unroll
  for (int r = 0; r < R; ++r) {
    const int gi = r0 + i0 + r;
    A.u[(size_t)gi * g.W + gj] = u[r];
    A.P1[(size_t)(gi + a) * g.W + gj] = p1[r];
    A.P2[(size_t)gi * W2 + gj + b] = p2[r];
  }
  if (i0 == 0 && s_top) A.out.ST[(size_t)(a - 1) * g.W + gj] = p1[0];
  if (j == 0 && s_lft) {
#pragma unroll
    for (int r = 0; r < R; ++r) A.out.SL[(size_t)(b - 1) * g.H + r0 + i0 + r] = p2[r];
  }
  if (last_row_here && s_bot) {
    A.P1[(size_t)(r0 + 128 + a) * g.W + gj] = pB;
    A.out.SB[(size_t)a * g.W + gj] = pB;
  }
  if (right_lane) {
    const int gi = r0 + i0 + j;
    const float pr = sPR[lr0 + j];
    A.P2[(size_t)gi * W2 + c0 + 128 + b] = pr;
    A.out.SR[(size_t)b * g.H + gi] = pr;
  }
}

// ---------------------------------------------------------------------------
// Warp-row kernel for exact 128 x 128 subdomains.  Warp w of a CTA owns R full rows
// of the tile (lane l holds columns 4l .. 4l+3 of each), so horizontal neighbours
// are in the lane's registers or one shuffle away, and the only data another warp
// needs are a warp's first-row pbar1 (read by the warp above) and last-row u (read
// by the warp below).  Those rows go through shared-memory slots, each guarded by
// an mbarrier that its single producer warp arrives on (all 32 lanes) and its
// single consumer warp waits on, so a warp only ever waits for its two vertical
// neighbours; no CTA-wide barrier runs inside the inner loop.  Rows crossing a CTA
// boundary are written into the neighbour CTA's slot (distributed shared memory)
// and signalled on its mbarrier with cluster-scope release.  Every wait is bounded:
// on timeout the kernel sets *err and carries on, so it always terminates.
//
// Why single-buffered slots are safe: a producer rewrites a slot one iteration
// later only after waiting on a signal that the slot's consumer sends after it read
// the slot (each half-step of a warp depends on the other half-step of the warp it
// feeds).
// A waiting warp sleeps in mbarrier.try_wait until the phase completes or the
// hardware's own time window ends (the hint is only an upper limit); kWaitLimit rounds
// of it bound the wait, at 3.8 ms measured on GB300 (dd_tv_fault_probe).
template <int R, int NW>
struct WrLayout {
  static constexpr int BAND = NW * R;
  static constexpr int SU = 0;                   // (NW + 1) x 128: slot w+1 = last-row u of warp w; slot 0 = row above
  static constexpr int SQ = SU + (NW + 1) * 128; // (NW + 1) x 128: slot w = first-row pbar1 of warp w; slot NW = row below
  static constexpr int CO = SQ + (NW + 1) * 128; // 64 x 8 coefficients
  static constexpr int MB = CO + 64 * 8;         // mbarriers (8 bytes each): mU[NW + 1], mQ[NW + 1]
  static constexpr size_t BYTES = sizeof(float) * MB + 8 * 2 * (NW + 1);
};

template <int R, int NW, int CL, int MINB, int FID, bool MASK>
__global__ void __launch_bounds__(32 * NW, MINB) k_fused_wr(const LocalArgs A) {
  using L = WrLayout<R, NW>;
  constexpr int BAND = L::BAND;
  static_assert(CL * BAND == 128, "a cluster covers the 128 rows of a tile");
  extern __shared__ __align__(16) float smem[];
  float* slotU = smem + L::SU;
  float* slotQ = smem + L::SQ;
  float* sCo = smem + L::CO;
  const uint32_t mbase = smem_addr(smem + L::MB);
  auto mU = [&](int q) { return mbase + 8u * q; };
  auto mQ = [&](int q) { return mbase + 8u * (NW + 1 + q); };

  const Grid g = A.g;
  const int rank = CL > 1 ? (int)blockIdx.x : 0;
  const int b = blockIdx.y, a = blockIdx.z;
  const int r0 = a * 128, c0 = b * 128;
  const bool s_top = a > 0, s_bot = a + 1 < g.NR, s_lft = b > 0, s_rgt = b + 1 < g.NC;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int i0 = rank * BAND + w * R;  // first tile row of this warp
  const int W2 = g.W + g.NC;
  const int jc = 4 * lane;             // first tile column of this lane
  const float tau = A.tau;
  const bool first_warp_of_tile = rank == 0 && w == 0;
  const bool last_warp_of_tile = rank == CL - 1 && w == NW - 1;
  const float lim_top = (first_warp_of_tile && !s_top) ? 0.f : 1.f;  // row 0 of the tile only
  const float lim_left = (lane == 0 && !s_lft) ? 0.f : 1.f;         // column 0 only
  const float lim_right = (lane == 31 && s_rgt) ? 1.f : 0.f;         // right side dofs (lane 31)
  // producers/consumers across the CTA boundary
  const bool push_down = CL > 1 && w == NW - 1 && rank + 1 < CL;   // my last row -> slot 0 of rank+1
  const bool push_up = CL > 1 && w == 0 && rank > 0;                 // my first row -> slot NW of rank-1
  uint32_t rem_slotU = 0, rem_mU = 0, rem_slotQ = 0, rem_mQ = 0;
  if (push_down) {
    rem_slotU = map_rank(smem_addr(slotU + jc), rank + 1);
    rem_mU = map_rank(mU(0), rank + 1);
  }
  if (push_up) {
    rem_slotQ = map_rank(smem_addr(slotQ + NW * 128 + jc), rank - 1);
    rem_mQ = map_rank(mQ(NW), rank - 1);
  }
  // does this warp wait for a producer before its u-step (row below) / p-step (row above)?
  const bool wait_below = !(last_warp_of_tile);  // last warp of the tile reads its own bottom-side slot
  const bool wait_above = !(rank == 0 && w == 0);

  // ---- set-up: barriers, coefficients
  if (threadIdx.x == 0) {
    for (int q = 0; q <= NW; ++q) {
      mbar_init(mU(q), 32);
      mbar_init(mQ(q), 32);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  for (int q = threadIdx.x; q < 8 * min(A.K, 64); q += 32 * NW) sCo[q] = reinterpret_cast<const float*>(A.coef)[q];
  if (rank == 0) {
    for (int q = threadIdx.x; q < 128; q += 32 * NW) slotU[q] = 0.f;  // u = 0 above the tile
  }

  // ---- load the state of rows i0 .. i0+R-1, columns jc .. jc+3
  float u[R][4], p1[R][4], p2[R][4], h1[R][4], h2[R][4], q1[R][4], q2[R][4], fg[R][4];
  float pR[R], hR[R], qR[R];
  float pB[4] = {0.f, 0.f, 0.f, 0.f}, hB[4] = {0.f, 0.f, 0.f, 0.f};
  uint32_t in_d = 0;
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const int gi = r0 + i0 + r;
    const size_t px = (size_t)gi * g.W + c0 + jc;
    const float4 uv = *reinterpret_cast<const float4*>(A.u + px);
    const float4 fv = *reinterpret_cast<const float4*>(A.f + px);
    const float4 pv = *reinterpret_cast<const float4*>(A.P1 + (size_t)(gi + a) * g.W + c0 + jc);
    const float uu[4] = {uv.x, uv.y, uv.z, uv.w}, ff[4] = {fv.x, fv.y, fv.z, fv.w}, pp[4] = {pv.x, pv.y, pv.z, pv.w};
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      u[r][c] = uu[c];
      float f = ff[c];
      if (FID == FID_SEG) f = (f - A.c1) * (f - A.c1) - (f - A.c2) * (f - A.c2);
      fg[r][c] = f;
      if (MASK && A.mask[px + c]) in_d |= 1u << (4 * r + c);
      p1[r][c] = pp[c];
      p2[r][c] = A.P2[(size_t)gi * W2 + c0 + b + jc + c];
      h1[r][c] = p1[r][c];
      h2[r][c] = p2[r][c];
      q1[r][c] = p1[r][c];
      q2[r][c] = p2[r][c];
    }
    pR[r] = hR[r] = 0.f;
    if (lane == 31 && s_rgt) {
      pR[r] = A.P2[(size_t)gi * W2 + c0 + b + 128];
      hR[r] = phat_s(pR[r], A.lamv[(size_t)b * g.H + gi], tau);
    }
    qR[r] = pR[r];
  }
  if (first_warp_of_tile && s_top) {
#pragma unroll
    for (int c = 0; c < 4; ++c) h1[0][c] = phat_t(p1[0][c], A.lamh[(size_t)(a - 1) * g.W + c0 + jc + c], tau);
  }
  if (lane == 0 && s_lft) {
#pragma unroll
    for (int r = 0; r < R; ++r) h2[r][0] = phat_t(p2[r][0], A.lamv[(size_t)(b - 1) * g.H + r0 + i0 + r], tau);
  }
  if (last_warp_of_tile && s_bot) {
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      pB[c] = A.P1[(size_t)(r0 + 128 + a) * g.W + c0 + jc + c];
      hB[c] = phat_s(pB[c], A.lamh[(size_t)a * g.W + c0 + jc + c], tau);
    }
  }
  // initial slots: first-row pbar1 of every warp, the tile's bottom side
  *reinterpret_cast<float4*>(slotQ + w * 128 + jc) = make_float4(q1[0][0], q1[0][1], q1[0][2], q1[0][3]);
  if (last_warp_of_tile) *reinterpret_cast<float4*>(slotQ + NW * 128 + jc) = make_float4(pB[0], pB[1], pB[2], pB[3]);
  __syncthreads();
  if (CL > 1) {
    cluster_arrive<true>();  // mbarrier inits of every CTA are visible before any remote arrive
    cluster_wait();
    if (push_up) st_cluster_v4(rem_slotQ, make_float4(q1[0][0], q1[0][1], q1[0][2], q1[0][3]));
    cluster_arrive<true>();
    cluster_wait();
  }

  bool timed_out = false;
  float* myU = slotU + (w + 1) * 128 + jc;   // last-row u of this warp (read by the warp below)
  const float* abU = slotU + w * 128 + jc;   // last-row u of the warp above
  float* myQ = slotQ + w * 128 + jc;         // first-row pbar1 of this warp (read by the warp above)
  const float* beQ = slotQ + (w + 1) * 128 + jc;  // first-row pbar1 of the warp below

  for (int k = 0; k < A.K; ++k) {
    const float4 ca = *reinterpret_cast<const float4*>(sCo + 8 * (k & 63));
    const float4 cb = *reinterpret_cast<const float4*>(sCo + 8 * (k & 63) + 4);
    Coef c{ca.x, ca.y, ca.z, ca.w, cb.x, cb.y, cb.z, cb.w};
    if (k >= 64) c = A.coef[k];
    // ---------------- u-step: needs the first-row pbar1 of the warp below (iteration k-1)
    if (k > 0 && wait_below && !mbar_wait(mQ(w + 1), (uint32_t)((k - 1) & 1))) timed_out = true;
    const float4 bq = *reinterpret_cast<const float4*>(beQ);
    const float below_last[4] = {bq.x, bq.y, bq.z, bq.w};
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const float nxt = __shfl_down_sync(0xffffffffu, q2[r][0], 1);
      const float right3 = lane == 31 ? qR[r] : nxt;
#pragma unroll
      for (int cc = 0; cc < 4; ++cc) {
        const float below = r + 1 < R ? q1[r + 1][cc] : below_last[cc];
        const float right = cc < 3 ? q2[r][cc + 1] : right3;
        const float d = div_px(q1[r][cc], below, q2[r][cc], right);
        u[r][cc] = u_update<FID>(u[r][cc], d, fg[r][cc], MASK && ((in_d >> (4 * r + cc)) & 1u), c);
      }
    }
    {
      const float4 lastu = make_float4(u[R - 1][0], u[R - 1][1], u[R - 1][2], u[R - 1][3]);
      if (push_down) {
        st_cluster_v4(rem_slotU, lastu);
        mbar_arrive_remote(rem_mU);
      } else {
        *reinterpret_cast<float4*>(myU) = lastu;
        mbar_arrive_local(mU(w + 1));
      }
    }
    // ---------------- p-step: needs the last-row u of the warp above (iteration k)
    if (wait_above && !mbar_wait(mU(w), (uint32_t)(k & 1))) timed_out = true;
    const float4 au = *reinterpret_cast<const float4*>(abU);
    const float above_first[4] = {au.x, au.y, au.z, au.w};
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const float prv = __shfl_up_sync(0xffffffffu, u[r][3], 1);
      const float left0 = lane == 0 ? 0.f : prv;
#pragma unroll
      for (int cc = 0; cc < 4; ++cc) {
        const float above = r > 0 ? u[r - 1][cc] : above_first[cc];
        p_update_lim(p1[r][cc], q1[r][cc], u[r][cc] - above, h1[r][cc], c, r == 0 ? lim_top : 1.f);
        const float left = cc > 0 ? u[r][cc - 1] : left0;
        p_update_lim(p2[r][cc], q2[r][cc], u[r][cc] - left, h2[r][cc], c, cc == 0 ? lim_left : 1.f);
      }
      p_update_lim(pR[r], qR[r], -u[r][3], hR[r], c, lim_right);  // right side (lane 31)
    }
    if (last_warp_of_tile && s_bot) {  // bottom side, read back by this warp's next u-step
      float qB[4];
#pragma unroll
      for (int cc = 0; cc < 4; ++cc) p_update(pB[cc], qB[cc], -u[R - 1][cc], hB[cc], c);
      *reinterpret_cast<float4*>(slotQ + NW * 128 + jc) = make_float4(qB[0], qB[1], qB[2], qB[3]);
      __syncwarp();
    }
    {
      const float4 firstq = make_float4(q1[0][0], q1[0][1], q1[0][2], q1[0][3]);
      if (push_up) {
        st_cluster_v4(rem_slotQ, firstq);
        mbar_arrive_remote(rem_mQ);
      } else {
        *reinterpret_cast<float4*>(myQ) = firstq;
        mbar_arrive_local(mQ(w));
      }
    }
  }
  if (timed_out) atomicOr(A.err, 1);
  if (CL > 1) {  // no CTA leaves while a neighbour may still write into its shared memory
    cluster_arrive<true>();
    cluster_wait();
  }

  // ---- store u^{n+1}, p~^{n+1} and the interface strips
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const int gi = r0 + i0 + r;
    const size_t px = (size_t)gi * g.W + c0 + jc;
    *reinterpret_cast<float4*>(A.u + px) = make_float4(u[r][0], u[r][1], u[r][2], u[r][3]);
    *reinterpret_cast<float4*>(A.P1 + (size_t)(gi + a) * g.W + c0 + jc) =
        make_float4(p1[r][0], p1[r][1], p1[r][2], p1[r][3]);
#pragma unroll
    for (int cc = 0; cc < 4; ++cc) A.P2[(size_t)gi * W2 + c0 + b + jc + cc] = p2[r][cc];
    if (lane == 31 && s_rgt) {
      A.P2[(size_t)gi * W2 + c0 + b + 128] = pR[r];
      A.out.SR[(size_t)b * g.H + gi] = pR[r];
    }
    if (lane == 0 && s_lft) A.out.SL[(size_t)(b - 1) * g.H + gi] = p2[r][0];
  }
  if (first_warp_of_tile && s_top)
    *reinterpret_cast<float4*>(A.out.ST + (size_t)(a - 1) * g.W + c0 + jc) =
        make_float4(p1[0][0], p1[0][1], p1[0][2], p1[0][3]);
  if (last_warp_of_tile && s_bot) {
    const float4 v = make_float4(pB[0], pB[1], pB[2], pB[3]);
    *reinterpret_cast<float4*>(A.P1 + (size_t)(r0 + 128 + a) * g.W + c0 + jc) = v;
    *reinterpret_cast<float4*>(A.out.SB + (size_t)a * g.W + c0 + jc) = v;
  }
}

// ---------------------------------------------------------------------------
// Full-tile kernel with asynchronous halo exchange.  Same arithmetic and mapping as
// k_fused_full, but inside the inner loop no cluster barrier runs: a halo row is
// written into the neighbour CTA with st.async, whose completion is counted (in
// bytes) on an mbarrier in the neighbour's shared memory, so the producing warps
// never wait for the remote store; only the warps that read a halo wait, on their
// own CTA's mbarrier (bounded).  Each halo mbarrier completes one phase per inner
// iteration: the consumer arrives once per phase with the expected byte count, the
// producer's stores bring the byte count to zero.  A producer cannot run a phase
// ahead of its consumer (its next halo row depends on the consumer's previous one),
// so the single halo buffers are never overwritten while being read.
template <int R, int TR>
struct AsyncLayout {
  using F = FullLayout<R, TR>;
  static constexpr int MB = (F::FLOATS + 1) & ~1;  // two mbarriers (8-byte aligned): u halo, pbar1 halo
  static constexpr size_t BYTES = sizeof(float) * MB + 16;
};

// Body of one CTA of the cluster that owns tile (a, b) of the image described by A.
template <int R, int TR, int CL, int FID, bool MASK>
__device__ __forceinline__ void fused_async_body(const LocalArgs& A, const int a, const int b) {
  using L = FullLayout<R, TR>;
  using AL = AsyncLayout<R, TR>;
  constexpr int BW = L::BW, BAND = L::BAND;
  static_assert(CL * BAND == 128 && CL > 1, "a cluster of CTAs covers the 128 rows of a tile");
  extern __shared__ __align__(16) float smem[];
  float* sU = smem + L::U;
  float* sQ2 = smem + L::Q2;
  float* sQ1 = smem + L::Q1;
  float* sF = smem + L::F;
  float* sPR = smem + L::PR;
  float* sHR = smem + L::HR;
  float* sCo = smem + L::CO;
  const uint32_t mbU = smem_addr(smem + AL::MB);      // u halo (row above the band) has landed
  const uint32_t mbQ = mbU + 8;                        // pbar1 halo (row below the band) has landed

  const Grid g = A.g;
  const int rank = (int)blockIdx.x;
  const int r0 = a * 128, c0 = b * 128;
  const bool s_top = a > 0, s_bot = a + 1 < g.NR, s_lft = b > 0, s_rgt = b + 1 < g.NC;
  const int j = threadIdx.x, ty = threadIdx.y;
  const int lr0 = ty * R;
  const int i0 = rank * BAND + lr0;
  const int W2 = g.W + g.NC;
  const int gj = c0 + j;
  const float tau = A.tau;
  const float lim_left = (j == 0 && !s_lft) ? 0.f : 1.f;
  const float lim_top = (i0 == 0 && !s_top) ? 0.f : 1.f;
  const bool last_row_here = rank == CL - 1 && ty == TR - 1;
  const bool push_down = ty == TR - 1 && rank + 1 < CL;  // my last row -> u halo of rank + 1
  const bool push_up = ty == 0 && rank > 0;              // my first row -> pbar1 halo of rank - 1
  const bool need_uh = ty == 0 && rank > 0;              // reads the u halo
  const bool need_qh = ty == TR - 1 && rank + 1 < CL;    // reads the pbar1 halo
  const bool right_lane = s_rgt && j < R;
  constexpr uint32_t kHaloBytes = 4 * BW;
  uint32_t remote_u = 0, remote_q1 = 0, remote_mbU = 0, remote_mbQ = 0;
  if (push_down) {
    remote_u = map_rank(smem_addr(sU + 1 + j), rank + 1);
    remote_mbU = map_rank(mbU, rank + 1);
  }
  if (push_up) {
    remote_q1 = map_rank(smem_addr(sQ1 + TR * BW + j), rank - 1);
    remote_mbQ = map_rank(mbQ, rank - 1);
  }
  if (j == 0 && ty == 0) {
    mbar_init(mbU, 1);
    mbar_init(mbQ, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }

  float u[R], p1[R], p2[R], h1[R], h2[R], q1[R];
  uint32_t in_d = 0;
  float pB = 0.f, hB = 0.f;

  for (int q = threadIdx.x + threadIdx.y * BW; q < 8 * min(A.K, L::kMaxSmemCoef); q += BW * TR)
    sCo[q] = reinterpret_cast<const float*>(A.coef)[q];
  if (rank == 0) sU[1 + j] = 0.f;
  if (j == 0) sU[0] = 0.f;
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const int gi = r0 + i0 + r;
    const size_t px = (size_t)gi * g.W + gj;
    u[r] = A.u[px];
    float fv = A.f[px];
    if (FID == FID_SEG) fv = (fv - A.c1) * (fv - A.c1) - (fv - A.c2) * (fv - A.c2);
    sF[(lr0 + r) * BW + j] = fv;
    if (MASK && A.mask[px]) in_d |= 1u << r;
    p1[r] = A.P1[(size_t)(gi + a) * g.W + gj];
    p2[r] = A.P2[(size_t)gi * W2 + gj + b];
    h1[r] = p1[r];
    h2[r] = p2[r];
    q1[r] = p1[r];
    sQ2[(lr0 + r) * L::QS + j] = p2[r];
    sU[(lr0 + r + 1) * L::US] = 0.f;
  }
  if (i0 == 0 && s_top) h1[0] = phat_t(p1[0], A.lamh[(size_t)(a - 1) * g.W + gj], tau);
  if (j == 0 && s_lft) {
#pragma unroll
    for (int r = 0; r < R; ++r) h2[r] = phat_t(p2[r], A.lamv[(size_t)(b - 1) * g.H + r0 + i0 + r], tau);
  }
  if (last_row_here) {
    if (s_bot) {
      pB = A.P1[(size_t)(r0 + 128 + a) * g.W + gj];
      hB = phat_s(pB, A.lamh[(size_t)a * g.W + gj], tau);
    }
    sQ1[TR * BW + j] = pB;
  }
  if (j < R) {
    float pr = 0.f, hr = 0.f;
    if (s_rgt) {
      const int gi = r0 + i0 + j;
      pr = A.P2[(size_t)gi * W2 + c0 + 128 + b];
      hr = phat_s(pr, A.lamv[(size_t)b * g.H + gi], tau);
    }
    sPR[lr0 + j] = pr;
    sHR[lr0 + j] = hr;
    sQ2[(lr0 + j) * L::QS + 128] = pr;
  }
  sQ1[ty * BW + j] = q1[0];
  __syncthreads();
  // every CTA's mbarriers are initialised before anyone signals them; the initial
  // pbar1 halo goes through a plain remote store ordered by the cluster barrier
  cluster_arrive<true>();
  cluster_wait();
  if (push_up) st_cluster(remote_q1, q1[0]);
  cluster_arrive<true>();
  cluster_wait();

  bool timed_out = false;
  float* sUr = sU + (lr0 + 1) * L::US + j + 1;
  float* sQ2r = sQ2 + lr0 * L::QS + j;
  const float* sFr = sF + lr0 * BW + j;

  for (int k = 0; k < A.K; ++k) {
    Coef c;
    if (k < L::kMaxSmemCoef) {
      const float4 ca = *reinterpret_cast<const float4*>(sCo + 8 * k);
      const float4 cb = *reinterpret_cast<const float4*>(sCo + 8 * k + 4);
      c = Coef{ca.x, ca.y, ca.z, ca.w, cb.x, cb.y, cb.z, cb.w};
    } else {
      c = A.coef[k];
    }
    // ---- u-step; the band's last row first (it feeds the CTA below)
    if (need_qh && k > 0) {  // pbar1 halo of iteration k-1
      if (j == 0) mbar_arrive_expect_tx(mbQ, kHaloBytes);
      if (!mbar_wait(mbQ, (uint32_t)((k - 1) & 1))) timed_out = true;
    }
#pragma unroll
    for (int rr = 0; rr < R; ++rr) {
      const int r = (rr + R - 1) % R;
      const float below = r + 1 < R ? q1[r + 1] : sQ1[(ty + 1) * BW + j];
      const float d = div_px(q1[r], below, sQ2r[r * L::QS], sQ2r[r * L::QS + 1]);
      u[r] = u_update<FID>(u[r], d, sFr[r * BW], MASK && ((in_d >> r) & 1u), c);
      sUr[r * L::US] = u[r];
      if (rr == 0 && push_down) st_async_f32(remote_u, u[R - 1], remote_mbU);
    }
    __syncthreads();
    // ---- p-step; the band's first row first (it feeds the CTA above)
    if (need_uh) {  // u halo of iteration k
      if (j == 0) mbar_arrive_expect_tx(mbU, kHaloBytes);
      if (!mbar_wait(mbU, (uint32_t)(k & 1))) timed_out = true;
    }
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const float above = r > 0 ? u[r - 1] : sUr[-L::US];
      p_update_lim(p1[r], q1[r], u[r] - above, h1[r], c, r == 0 ? lim_top : 1.f);
      float q2;
      p_update_lim(p2[r], q2, u[r] - sUr[r * L::US - 1], h2[r], c, lim_left);
      sQ2r[r * L::QS] = q2;
      if (r == 0) {
        sQ1[ty * BW + j] = q1[0];
        if (push_up) st_async_f32(remote_q1, q1[0], remote_mbQ);
      }
    }
    if (last_row_here && s_bot) {
      float qB;
      p_update(pB, qB, -u[R - 1], hB, c);
      sQ1[TR * BW + j] = qB;
    }
    if (right_lane) {
      const int lr = lr0 + j;
      float pr = sPR[lr], qr;
      p_update(pr, qr, -sU[(lr + 1) * L::US + 128], sHR[lr], c);
      sPR[lr] = pr;
      sQ2[lr * L::QS + 128] = qr;
    }
    __syncthreads();
  }
  // the last pbar1 halo is never read: wait for it to land before leaving
  if (need_qh && A.K > 0) {
    if (j == 0) mbar_arrive_expect_tx(mbQ, kHaloBytes);
    if (!mbar_wait(mbQ, (uint32_t)((A.K - 1) & 1))) timed_out = true;
  }
  if (timed_out) atomicOr(A.err, 1);
  cluster_arrive<true>();
  cluster_wait();

#pragma unroll
  for (int r = 0; r < R; ++r) {
    const int gi = r0 + i0 + r;
    A.u[(size_t)gi * g.W + gj] = u[r];
    A.P1[(size_t)(gi + a) * g.W + gj] = p1[r];
    A.P2[(size_t)gi * W2 + gj + b] = p2[r];
  }
  if (i0 == 0 && s_top) A.out.ST[(size_t)(a - 1) * g.W + gj] = p1[0];
  if (j == 0 && s_lft) {
#pragma unroll
    for (int r = 0; r < R; ++r) A.out.SL[(size_t)(b - 1) * g.H + r0 + i0 + r] = p2[r];
  }
  if (last_row_here && s_bot) {
    A.P1[(size_t)(r0 + 128 + a) * g.W + gj] = pB;
    A.out.SB[(size_t)a * g.W + gj] = pB;
  }
  if (right_lane) {
    const int gi = r0 + i0 + j;
    const float pr = sPR[lr0 + j];
    A.P2[(size_t)gi * W2 + c0 + 128 + b] = pr;
    A.out.SR[(size_t)b * g.H + gi] = pr;
  }
}

template <int R, int TR, int CL, int MINB, int FID, bool MASK>
__global__ void __launch_bounds__(128 * TR, MINB) k_fused_async(const LocalArgs A) {
  fused_async_body<R, TR, CL, FID, MASK>(A, blockIdx.z, blockIdx.y);
}

// Batched launch: blockIdx.y enumerates the tiles of every image of a batch; each
// image has its own descriptor (geometry, buffers, fidelity, steps).
template <int R, int TR, int CL, int MINB>
__global__ void __launch_bounds__(128 * TR, MINB) k_fused_async_batch(const BatchArgs B) {
  const int t = blockIdx.y;
  const int img = B.tile_img[t];
  LocalArgs A = B.args[img];
  A.out = B.strips[2 * img + B.write_set];
  const int lt = t - B.tile_base[img];
  const int a = lt / A.g.NC, b = lt - a * A.g.NC;
  switch (B.fid[img]) {
    case FID_L2: fused_async_body<R, TR, CL, FID_L2, false>(A, a, b); break;
    case FID_L1: fused_async_body<R, TR, CL, FID_L1, false>(A, a, b); break;
    default: fused_async_body<R, TR, CL, FID_SEG, false>(A, a, b); break;
  }
}

// ---------------------------------------------------------------------------
// Persistent asynchronous kernel.  The arithmetic and on-chip mapping of
// k_fused_async, but each cluster loops over subdomains t = cluster, cluster + C, ...
// While it iterates on one subdomain, every thread prefetches the values it will own
// in the next one into shared memory (cp.async), so state loads overlap the inner
// loop.  The two halo mbarriers live for the whole kernel; their phases are counted
// across subdomains (K phases each per subdomain).  A consumer re-arms the next phase
// (arrive.expect_tx) as soon as its wait on the current one completes; every halo a
// producer sends depends on data the consumer sent after re-arming, so bytes always
// land in the armed phase.  No barrier separates consecutive subdomains: the initial
// pbar1 halo row is ordinary state and is prefetched from global memory, and the
// warps that send a CTA's halos are the ones that drain (wait for) the last halo they
// receive, which their neighbour sends only after reading the halo they sent before,
// so no halo buffer is overwritten while it may still be read.

// PK: the inner loop works on packed pairs of rows (r, r + R/2) with `*.f32x2`
// arithmetic (same bits as the scalar loop; the clamps stay scalar).
template <int R, int TR, int CL, int FID, bool MASK, bool PK>
__device__ __forceinline__ void fused_pa_body(const LocalArgs& A, const int first, const int stride) {
  using L = FullLayout<R, TR>;
  using P = PaLayout<R, TR>;
  constexpr int BW = L::BW, BAND = L::BAND, NT = P::NT;
  static_assert(CL * BAND == 128 && CL > 1, "a cluster of CTAs covers the 128 rows of a tile");
  extern __shared__ __align__(16) float smem[];
  float* sU = smem + L::U;
  float* sQ2 = smem + L::Q2;
  float* sQ1 = smem + L::Q1;
  float* sF = smem + L::F;
  float* sPR = smem + L::PR;
  float* sHR = smem + L::HR;
  float* sCo = smem + L::CO;
  float* stg = smem + P::ST;
  float* stx = smem + P::SX;
  const uint32_t mbU = smem_addr(smem + P::MB);
  const uint32_t mbQ = mbU + 8;

  const Grid g = A.g;
  const int T = g.NR * g.NC;
  const int rank = (int)blockIdx.x;
  const int j = threadIdx.x, ty = threadIdx.y;
  const int tid = ty * BW + j;
  const int lr0 = ty * R;
  const int i0 = rank * BAND + lr0;
  const int W2 = g.W + g.NC;
  const float tau = A.tau;
  const int K = A.K;
  const bool last_row_here = rank == CL - 1 && ty == TR - 1;
  const bool push_down = ty == TR - 1 && rank + 1 < CL;
  const bool push_up = ty == 0 && rank > 0;
  const bool need_uh = ty == 0 && rank > 0;
  const bool need_qh = ty == TR - 1 && rank + 1 < CL;
  constexpr uint32_t kHaloBytes = 4 * BW;
  uint32_t remote_u = 0, remote_q1 = 0, remote_mbU = 0, remote_mbQ = 0;
  if (push_down) {
    remote_u = map_rank(smem_addr(sU + 1 + j), rank + 1);
    remote_mbU = map_rank(mbU, rank + 1);
  }
  if (push_up) {
    remote_q1 = map_rank(smem_addr(sQ1 + TR * BW + j), rank - 1);
    remote_mbQ = map_rank(mbQ, rank - 1);
  }
  if (tid == 0) {
    mbar_init(mbU, 1);
    mbar_init(mbQ, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  for (int q = tid; q < 8 * min(K, L::kMaxSmemCoef); q += NT) sCo[q] = reinterpret_cast<const float*>(A.coef)[q];
  if (rank == 0) sU[1 + j] = 0.f;  // u = 0 above every tile's first row
  if (j == 0) sU[0] = 0.f;
  __syncthreads();
  // arm the first phase of each halo barrier this CTA consumes
  if (need_uh && j == 0) mbar_arrive_expect_tx(mbU, kHaloBytes);
  if (need_qh && j == 0) mbar_arrive_expect_tx(mbQ, kHaloBytes);
  cluster_arrive<true>();  // barriers initialised and armed everywhere before any halo is sent
  cluster_wait();

  auto prefetch = [&](int t) {
    const int a = t / g.NC, b = t - a * g.NC;
    const int r0 = a * 128, c0 = b * 128, gj = c0 + j;
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const int gi = r0 + i0 + r;
      cp_async4(stg + (0 * R + r) * NT + tid, A.u + (size_t)gi * g.W + gj);
      cp_async4(stg + (1 * R + r) * NT + tid, A.f + (size_t)gi * g.W + gj);
      cp_async4(stg + (2 * R + r) * NT + tid, A.P1 + (size_t)(gi + a) * g.W + gj);
      cp_async4(stg + (3 * R + r) * NT + tid, A.P2 + (size_t)gi * W2 + gj + b);
    }
    if (i0 == 0 && a > 0) cp_async4(stx + 0 * NT + tid, A.lamh + (size_t)(a - 1) * g.W + gj);
    if (last_row_here && a + 1 < g.NR) {
      cp_async4(stx + 1 * NT + tid, A.P1 + (size_t)(r0 + 128 + a) * g.W + gj);
      cp_async4(stx + 2 * NT + tid, A.lamh + (size_t)a * g.W + gj);
    }
    if (j == 0 && b > 0) {
#pragma unroll
      for (int r = 0; r < R; ++r) cp_async4(stx + (3 + r) * NT + tid, A.lamv + (size_t)(b - 1) * g.H + r0 + i0 + r);
    }
    if (j < R && b + 1 < g.NC) {
      const int gi = r0 + i0 + j;
      cp_async4(stx + (3 + R) * NT + tid, A.P2 + (size_t)gi * W2 + c0 + 128 + b);
      cp_async4(stx + (4 + R) * NT + tid, A.lamv + (size_t)b * g.H + gi);
    }
    if (need_qh) cp_async4(stx + (5 + R) * NT + tid, A.P1 + (size_t)(r0 + i0 + R + a) * g.W + gj);
    cp_async_commit();
  };

  bool timed_out = false;
  uint32_t phU = 0, phQ = 0;  // index of the next phase of mbU / mbQ this CTA waits for
  auto wait_u = [&]() {
    if (!mbar_wait(mbU, phU & 1)) timed_out = true;
    ++phU;
    if (j == 0) mbar_arrive_expect_tx(mbU, kHaloBytes);  // arm the next phase
  };
  auto wait_q = [&]() {
    if (!mbar_wait(mbQ, phQ & 1)) timed_out = true;
    ++phQ;
    if (j == 0) mbar_arrive_expect_tx(mbQ, kHaloBytes);
  };

  float* sUr = sU + (lr0 + 1) * L::US + j + 1;
  float* sQ2r = sQ2 + lr0 * L::QS + j;
  const float* sFr = sF + lr0 * BW + j;
  if (first < T) prefetch(first);

  for (int t = first; t < T; t += stride) {
    const int a = t / g.NC, b = t - a * g.NC;
    const int r0 = a * 128, c0 = b * 128, gj = c0 + j;
    const bool s_top = a > 0, s_bot = a + 1 < g.NR, s_lft = b > 0, s_rgt = b + 1 < g.NC;
    const float lim_left = (j == 0 && !s_lft) ? 0.f : 1.f;
    const float lim_top = (i0 == 0 && !s_top) ? 0.f : 1.f;
    const bool right_lane = s_rgt && j < R;
    float u[R], p1[R], p2[R], h1[R], h2[R], q1[R];
    uint32_t in_d = 0;
    float pB = 0.f, hB = 0.f;

    cp_async_wait_all();
    __syncthreads();  // staging landed; the previous subdomain's shared arrays are free
#pragma unroll
    for (int r = 0; r < R; ++r) {
      u[r] = stg[(0 * R + r) * NT + tid];
      float fv = stg[(1 * R + r) * NT + tid];
      if (FID == FID_SEG) fv = (fv - A.c1) * (fv - A.c1) - (fv - A.c2) * (fv - A.c2);
      sF[(lr0 + r) * BW + j] = fv;
      if (MASK && A.mask[(size_t)(r0 + i0 + r) * g.W + gj]) in_d |= 1u << r;
      p1[r] = stg[(2 * R + r) * NT + tid];
      p2[r] = stg[(3 * R + r) * NT + tid];
      h1[r] = p1[r];
      h2[r] = p2[r];
      q1[r] = p1[r];
      sQ2[(lr0 + r) * L::QS + j] = p2[r];
      sU[(lr0 + r + 1) * L::US] = 0.f;
    }
    if (i0 == 0 && s_top) h1[0] = phat_t(p1[0], stx[0 * NT + tid], tau);
    if (j == 0 && s_lft) {
#pragma unroll
      for (int r = 0; r < R; ++r) h2[r] = phat_t(p2[r], stx[(3 + r) * NT + tid], tau);
    }
    if (last_row_here) {
      if (s_bot) {
        pB = stx[1 * NT + tid];
        hB = phat_s(pB, stx[2 * NT + tid], tau);
      }
      sQ1[TR * BW + j] = pB;
    }
    if (need_qh) sQ1[TR * BW + j] = stx[(5 + R) * NT + tid];  // first row of the band below
    if (j < R) {
      float pr = 0.f, hr = 0.f;
      if (s_rgt) {
        pr = stx[(3 + R) * NT + tid];
        hr = phat_s(pr, stx[(4 + R) * NT + tid], tau);
      }
      sPR[lr0 + j] = pr;
      sHR[lr0 + j] = hr;
      sQ2[(lr0 + j) * L::QS + 128] = pr;
    }
    sQ1[ty * BW + j] = q1[0];
    __syncthreads();  // staging consumed by every thread
    if (t + stride < T) prefetch(t + stride);

    if constexpr (PK) {
      constexpr int H2 = R / 2;
      static_assert(R % 2 == 0, "rows are paired");
      f32x2 U[H2], P1v[H2], P2v[H2], H1v[H2], H2v[H2], Q1v[H2];
#pragma unroll
      for (int i = 0; i < H2; ++i) {
        U[i] = pk2(u[i], u[i + H2]);
        P1v[i] = pk2(p1[i], p1[i + H2]);
        P2v[i] = pk2(p2[i], p2[i + H2]);
        H1v[i] = pk2(h1[i], h1[i + H2]);
        H2v[i] = pk2(h2[i], h2[i + H2]);
        Q1v[i] = pk2(q1[i], q1[i + H2]);
      }
      for (int k = 0; k < K; ++k) {
        Coef c;
        if (k < L::kMaxSmemCoef) {
          const float4 ca = *reinterpret_cast<const float4*>(sCo + 8 * k);
          const float4 cb = *reinterpret_cast<const float4*>(sCo + 8 * k + 4);
          c = Coef{ca.x, ca.y, ca.z, ca.w, cb.x, cb.y, cb.z, cb.w};
        } else {
          c = A.coef[k];
        }
        const f32x2 SIG = pk2(c.sig, c.sig), UA = pk2(c.ua, c.ua), UB = pk2(c.ub, c.ub);
        const f32x2 PA = pk2(c.pa, c.pa), PC = pk2(c.pc, c.pc), PB = pk2(c.pb, c.pb), TH = pk2(c.th, c.th);
        if (need_qh && k > 0) wait_q();  // pbar1 halo of iteration k-1
        // u-step on row pairs; the pair holding the band's last row first
#pragma unroll
        for (int ii = 0; ii < H2; ++ii) {
          const int i = (ii + H2 - 1) % H2;
          const f32x2 below = i + 1 < H2 ? Q1v[i + 1] : pk2(hi2(Q1v[0]), sQ1[(ty + 1) * BW + j]);
          const f32x2 left = pk2(sQ2r[i * L::QS], sQ2r[(i + H2) * L::QS]);
          const f32x2 right = pk2(sQ2r[i * L::QS + 1], sQ2r[(i + H2) * L::QS + 1]);
          const f32x2 d = sub2(add2(sub2(below, Q1v[i]), right), left);  // div_px
          const f32x2 fg = pk2(sFr[i * BW], sFr[(i + H2) * BW]);
          const f32x2 ub = fma2(SIG, d, U[i]);
          f32x2 un;
          if (FID == FID_L2) {
            un = fma2(UB, fg, mul2(UA, ub));
            if (MASK)
              un = pk2(((in_d >> i) & 1u) ? lo2(ub) : lo2(un), ((in_d >> (i + H2)) & 1u) ? hi2(ub) : hi2(un));
          } else {
            un = pk2(prox_ubar<FID>(lo2(ub), lo2(fg), MASK && ((in_d >> i) & 1u), c),
                     prox_ubar<FID>(hi2(ub), hi2(fg), MASK && ((in_d >> (i + H2)) & 1u), c));
          }
          U[i] = un;
          sUr[i * L::US] = lo2(un);
          sUr[(i + H2) * L::US] = hi2(un);
          if (ii == 0 && push_down) st_async_f32(remote_u, hi2(un), remote_mbU);
        }
        __syncthreads();
        if (need_uh) wait_u();  // u halo of iteration k
        // p-step on row pairs; the pair holding the band's first row first
#pragma unroll
        for (int i = 0; i < H2; ++i) {
          const f32x2 above = i > 0 ? U[i - 1] : pk2(sUr[-L::US], lo2(U[H2 - 1]));
          const f32x2 leftu = pk2(sUr[i * L::US - 1], sUr[(i + H2) * L::US - 1]);
          {
            const f32x2 tt = fma2(PC, sub2(U[i], above), fma2(PA, P1v[i], mul2(PB, H1v[i])));  // p_target
            const float l0 = i == 0 ? lim_top : 1.f;
            const f32x2 pn = pk2(fminf(fmaxf(lo2(tt), -l0), l0), fminf(fmaxf(hi2(tt), -1.f), 1.f));
            Q1v[i] = fma2(TH, sub2(pn, P1v[i]), pn);
            P1v[i] = pn;
          }
          {
            const f32x2 tt = fma2(PC, sub2(U[i], leftu), fma2(PA, P2v[i], mul2(PB, H2v[i])));
            const f32x2 pn = pk2(fminf(fmaxf(lo2(tt), -lim_left), lim_left),
                                 fminf(fmaxf(hi2(tt), -lim_left), lim_left));
            const f32x2 q2 = fma2(TH, sub2(pn, P2v[i]), pn);
            P2v[i] = pn;
            sQ2r[i * L::QS] = lo2(q2);
            sQ2r[(i + H2) * L::QS] = hi2(q2);
          }
          if (i == 0) {
            const float q10 = lo2(Q1v[0]);
            sQ1[ty * BW + j] = q10;
            if (push_up) st_async_f32(remote_q1, q10, remote_mbQ);
          }
        }
        if (last_row_here && s_bot) {
          float qB;
          p_update(pB, qB, -hi2(U[H2 - 1]), hB, c);
          sQ1[TR * BW + j] = qB;
        }
        if (right_lane) {
          const int lr = lr0 + j;
          float pr = sPR[lr], qr;
          p_update(pr, qr, -sU[(lr + 1) * L::US + 128], sHR[lr], c);
          sPR[lr] = pr;
          sQ2[lr * L::QS + 128] = qr;
        }
        __syncthreads();
      }
#pragma unroll
      for (int i = 0; i < H2; ++i) {
        u[i] = lo2(U[i]);
        u[i + H2] = hi2(U[i]);
        p1[i] = lo2(P1v[i]);
        p1[i + H2] = hi2(P1v[i]);
        p2[i] = lo2(P2v[i]);
        p2[i + H2] = hi2(P2v[i]);
      }
    } else {
      for (int k = 0; k < K; ++k) {
        Coef c;
        if (k < L::kMaxSmemCoef) {
          const float4 ca = *reinterpret_cast<const float4*>(sCo + 8 * k);
          const float4 cb = *reinterpret_cast<const float4*>(sCo + 8 * k + 4);
          c = Coef{ca.x, ca.y, ca.z, ca.w, cb.x, cb.y, cb.z, cb.w};
        } else {
          c = A.coef[k];
        }
        if (need_qh && k > 0) wait_q();  // pbar1 halo of iteration k-1
  #pragma unroll
        for (int rr = 0; rr < R; ++rr) {
          const int r = (rr + R - 1) % R;
          const float below = r + 1 < R ? q1[r + 1] : sQ1[(ty + 1) * BW + j];
          const float d = div_px(q1[r], below, sQ2r[r * L::QS], sQ2r[r * L::QS + 1]);
          u[r] = u_update<FID>(u[r], d, sFr[r * BW], MASK && ((in_d >> r) & 1u), c);
          sUr[r * L::US] = u[r];
          if (rr == 0 && push_down) st_async_f32(remote_u, u[R - 1], remote_mbU);
        }
        __syncthreads();
        if (need_uh) wait_u();  // u halo of iteration k
  #pragma unroll
        for (int r = 0; r < R; ++r) {
          const float above = r > 0 ? u[r - 1] : sUr[-L::US];
          p_update_lim(p1[r], q1[r], u[r] - above, h1[r], c, r == 0 ? lim_top : 1.f);
          float q2;
          p_update_lim(p2[r], q2, u[r] - sUr[r * L::US - 1], h2[r], c, lim_left);
          sQ2r[r * L::QS] = q2;
          if (r == 0) {
            sQ1[ty * BW + j] = q1[0];
            if (push_up) st_async_f32(remote_q1, q1[0], remote_mbQ);
          }
        }
        if (last_row_here && s_bot) {
          float qB;
          p_update(pB, qB, -u[R - 1], hB, c);
          sQ1[TR * BW + j] = qB;
        }
        if (right_lane) {
          const int lr = lr0 + j;
          float pr = sPR[lr], qr;
          p_update(pr, qr, -sU[(lr + 1) * L::US + 128], sHR[lr], c);
          sPR[lr] = pr;
          sQ2[lr * L::QS + 128] = qr;
        }
        __syncthreads();
      }
    }
    if (need_qh) wait_q();  // drain the last pbar1 halo (not read)

#pragma unroll
    for (int r = 0; r < R; ++r) {
      const int gi = r0 + i0 + r;
      A.u[(size_t)gi * g.W + gj] = u[r];
      A.P1[(size_t)(gi + a) * g.W + gj] = p1[r];
      A.P2[(size_t)gi * W2 + gj + b] = p2[r];
    }
    if (i0 == 0 && s_top) A.out.ST[(size_t)(a - 1) * g.W + gj] = p1[0];
    if (j == 0 && s_lft) {
#pragma unroll
      for (int r = 0; r < R; ++r) A.out.SL[(size_t)(b - 1) * g.H + r0 + i0 + r] = p2[r];
    }
    if (last_row_here && s_bot) {
      A.P1[(size_t)(r0 + 128 + a) * g.W + gj] = pB;
      A.out.SB[(size_t)a * g.W + gj] = pB;
    }
    if (right_lane) {
      const int gi = r0 + i0 + j;
      const float pr = sPR[lr0 + j];
      A.P2[(size_t)gi * W2 + c0 + 128 + b] = pr;
      A.out.SR[(size_t)b * g.H + gi] = pr;
    }
  }
  cp_async_wait_all();
  cluster_arrive<true>();  // no CTA leaves while a neighbour may still write into it
  cluster_wait();
  if (timed_out) atomicOr(A.err, 1);
}

// Persistent body over a source of subdomains of several images (the batch): the
// single-image body above with, per subdomain, the image's geometry, parameters,
// strips and fidelity (dispatched at run time), and the image's coefficients reloaded
// into shared memory when the image changes.  (The single-image kernel keeps its own
// copy of the body: the per-subdomain indirection measured 2 % slower there.)
template <int R, int TR, int CL, bool MASK, bool PK, class Src>
__device__ __forceinline__ void fused_pa_run(const Src& S, const int first, const int stride) {
  using L = FullLayout<R, TR>;
  using P = PaLayout<R, TR>;
  constexpr int BW = L::BW, BAND = L::BAND, NT = P::NT;
  static_assert(CL * BAND == 128 && CL > 1, "a cluster of CTAs covers the 128 rows of a tile");
  extern __shared__ __align__(16) float smem[];
  float* sU = smem + L::U;
  float* sQ2 = smem + L::Q2;
  float* sQ1 = smem + L::Q1;
  float* sF = smem + L::F;
  float* sPR = smem + L::PR;
  float* sHR = smem + L::HR;
  float* sCo = smem + L::CO;
  float* stg = smem + P::ST;
  float* stx = smem + P::SX;
  const uint32_t mbU = smem_addr(smem + P::MB);
  const uint32_t mbQ = mbU + 8;

  const int T = S.count();
  const int rank = (int)blockIdx.x;
  const int j = threadIdx.x, ty = threadIdx.y;
  const int tid = ty * BW + j;
  const int lr0 = ty * R;
  const int i0 = rank * BAND + lr0;
  const int K = S.inner();
  const bool last_row_here = rank == CL - 1 && ty == TR - 1;
  const bool push_down = ty == TR - 1 && rank + 1 < CL;
  const bool push_up = ty == 0 && rank > 0;
  const bool need_uh = ty == 0 && rank > 0;
  const bool need_qh = ty == TR - 1 && rank + 1 < CL;
  constexpr uint32_t kHaloBytes = 4 * BW;
  uint32_t remote_u = 0, remote_q1 = 0, remote_mbU = 0, remote_mbQ = 0;
  if (push_down) {
    remote_u = map_rank(smem_addr(sU + 1 + j), rank + 1);
    remote_mbU = map_rank(mbU, rank + 1);
  }
  if (push_up) {
    remote_q1 = map_rank(smem_addr(sQ1 + TR * BW + j), rank - 1);
    remote_mbQ = map_rank(mbQ, rank - 1);
  }
  if (tid == 0) {
    mbar_init(mbU, 1);
    mbar_init(mbQ, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  int cur_img = -1;  // image whose coefficients are in sCo
  if (rank == 0) sU[1 + j] = 0.f;  // u = 0 above every tile's first row
  if (j == 0) sU[0] = 0.f;
  __syncthreads();
  // arm the first phase of each halo barrier this CTA consumes
  if (need_uh && j == 0) mbar_arrive_expect_tx(mbU, kHaloBytes);
  if (need_qh && j == 0) mbar_arrive_expect_tx(mbQ, kHaloBytes);
  cluster_arrive<true>();  // barriers initialised and armed everywhere before any halo is sent
  cluster_wait();

  auto prefetch = [&](int t) {
    const LocalArgs& A = S.args(t);
    const Grid g = A.g;
    const int W2 = g.W + g.NC;
    const int lt = S.local(t);
    const int a = lt / g.NC, b = lt - a * g.NC;
    const int r0 = a * 128, c0 = b * 128, gj = c0 + j;
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const int gi = r0 + i0 + r;
      cp_async4(stg + (0 * R + r) * NT + tid, A.u + (size_t)gi * g.W + gj);
      cp_async4(stg + (1 * R + r) * NT + tid, A.f + (size_t)gi * g.W + gj);
      cp_async4(stg + (2 * R + r) * NT + tid, A.P1 + (size_t)(gi + a) * g.W + gj);
      cp_async4(stg + (3 * R + r) * NT + tid, A.P2 + (size_t)gi * W2 + gj + b);
    }
    if (i0 == 0 && a > 0) cp_async4(stx + 0 * NT + tid, A.lamh + (size_t)(a - 1) * g.W + gj);
    if (last_row_here && a + 1 < g.NR) {
      cp_async4(stx + 1 * NT + tid, A.P1 + (size_t)(r0 + 128 + a) * g.W + gj);
      cp_async4(stx + 2 * NT + tid, A.lamh + (size_t)a * g.W + gj);
    }
    if (j == 0 && b > 0) {
#pragma unroll
      for (int r = 0; r < R; ++r) cp_async4(stx + (3 + r) * NT + tid, A.lamv + (size_t)(b - 1) * g.H + r0 + i0 + r);
    }
    if (j < R && b + 1 < g.NC) {
      const int gi = r0 + i0 + j;
      cp_async4(stx + (3 + R) * NT + tid, A.P2 + (size_t)gi * W2 + c0 + 128 + b);
      cp_async4(stx + (4 + R) * NT + tid, A.lamv + (size_t)b * g.H + gi);
    }
    if (need_qh) cp_async4(stx + (5 + R) * NT + tid, A.P1 + (size_t)(r0 + i0 + R + a) * g.W + gj);
    cp_async_commit();
  };

  bool timed_out = false;
  uint32_t phU = 0, phQ = 0;  // index of the next phase of mbU / mbQ this CTA waits for
  auto wait_u = [&]() {
    if (!mbar_wait(mbU, phU & 1)) timed_out = true;
    ++phU;
    if (j == 0) mbar_arrive_expect_tx(mbU, kHaloBytes);  // arm the next phase
  };
  auto wait_q = [&]() {
    if (!mbar_wait(mbQ, phQ & 1)) timed_out = true;
    ++phQ;
    if (j == 0) mbar_arrive_expect_tx(mbQ, kHaloBytes);
  };

  float* sUr = sU + (lr0 + 1) * L::US + j + 1;
  float* sQ2r = sQ2 + lr0 * L::QS + j;
  const float* sFr = sF + lr0 * BW + j;
  if (first < T) prefetch(first);

  for (int t = first; t < T; t += stride) {
    const int img = S.image(t);
    const LocalArgs& A = S.args(t);
    const Grid g = A.g;
    const int W2 = g.W + g.NC;
    const float tau = A.tau;
    const int lt = S.local(t);
    const int a = lt / g.NC, b = lt - a * g.NC;
    const int r0 = a * 128, c0 = b * 128, gj = c0 + j;
    const bool s_top = a > 0, s_bot = a + 1 < g.NR, s_lft = b > 0, s_rgt = b + 1 < g.NC;
    const float lim_left = (j == 0 && !s_lft) ? 0.f : 1.f;
    const float lim_top = (i0 == 0 && !s_top) ? 0.f : 1.f;
    const bool right_lane = s_rgt && j < R;

    cp_async_wait_all();
    __syncthreads();  // staging landed; the previous subdomain's shared arrays are free
    if (img != cur_img) {  // made visible by the barrier after the unpack
      for (int q = tid; q < 8 * min(K, L::kMaxSmemCoef); q += NT) sCo[q] = reinterpret_cast<const float*>(A.coef)[q];
      cur_img = img;
    }
    auto tile_body = [&](auto fidc) {
    constexpr int FID = decltype(fidc)::value;
    float u[R], p1[R], p2[R], h1[R], h2[R], q1[R];
    uint32_t in_d = 0;
    float pB = 0.f, hB = 0.f;
#pragma unroll
    for (int r = 0; r < R; ++r) {
      u[r] = stg[(0 * R + r) * NT + tid];
      float fv = stg[(1 * R + r) * NT + tid];
      if (FID == FID_SEG) fv = (fv - A.c1) * (fv - A.c1) - (fv - A.c2) * (fv - A.c2);
      sF[(lr0 + r) * BW + j] = fv;
      if (MASK && A.mask[(size_t)(r0 + i0 + r) * g.W + gj]) in_d |= 1u << r;
      p1[r] = stg[(2 * R + r) * NT + tid];
      p2[r] = stg[(3 * R + r) * NT + tid];
      h1[r] = p1[r];
      h2[r] = p2[r];
      q1[r] = p1[r];
      sQ2[(lr0 + r) * L::QS + j] = p2[r];
      sU[(lr0 + r + 1) * L::US] = 0.f;
    }
    if (i0 == 0 && s_top) h1[0] = phat_t(p1[0], stx[0 * NT + tid], tau);
    if (j == 0 && s_lft) {
#pragma unroll
      for (int r = 0; r < R; ++r) h2[r] = phat_t(p2[r], stx[(3 + r) * NT + tid], tau);
    }
    if (last_row_here) {
      if (s_bot) {
        pB = stx[1 * NT + tid];
        hB = phat_s(pB, stx[2 * NT + tid], tau);
      }
      sQ1[TR * BW + j] = pB;
    }
    if (need_qh) sQ1[TR * BW + j] = stx[(5 + R) * NT + tid];  // first row of the band below
    if (j < R) {
      float pr = 0.f, hr = 0.f;
      if (s_rgt) {
        pr = stx[(3 + R) * NT + tid];
        hr = phat_s(pr, stx[(4 + R) * NT + tid], tau);
      }
      sPR[lr0 + j] = pr;
      sHR[lr0 + j] = hr;
      sQ2[(lr0 + j) * L::QS + 128] = pr;
    }
    sQ1[ty * BW + j] = q1[0];
    __syncthreads();  // staging consumed by every thread
    if (t + stride < T) prefetch(t + stride);

    if constexpr (PK) {
      constexpr int H2 = R / 2;
      static_assert(R % 2 == 0, "rows are paired");
      f32x2 U[H2], P1v[H2], P2v[H2], H1v[H2], H2v[H2], Q1v[H2];
#pragma unroll
      for (int i = 0; i < H2; ++i) {
        U[i] = pk2(u[i], u[i + H2]);
        P1v[i] = pk2(p1[i], p1[i + H2]);
        P2v[i] = pk2(p2[i], p2[i + H2]);
        H1v[i] = pk2(h1[i], h1[i + H2]);
        H2v[i] = pk2(h2[i], h2[i + H2]);
        Q1v[i] = pk2(q1[i], q1[i + H2]);
      }
      for (int k = 0; k < K; ++k) {
        Coef c;
        if (k < L::kMaxSmemCoef) {
          const float4 ca = *reinterpret_cast<const float4*>(sCo + 8 * k);
          const float4 cb = *reinterpret_cast<const float4*>(sCo + 8 * k + 4);
          c = Coef{ca.x, ca.y, ca.z, ca.w, cb.x, cb.y, cb.z, cb.w};
        } else {
          c = A.coef[k];
        }
        const f32x2 SIG = pk2(c.sig, c.sig), UA = pk2(c.ua, c.ua), UB = pk2(c.ub, c.ub);
        const f32x2 PA = pk2(c.pa, c.pa), PC = pk2(c.pc, c.pc), PB = pk2(c.pb, c.pb), TH = pk2(c.th, c.th);
        if (need_qh && k > 0) wait_q();  // pbar1 halo of iteration k-1
        // u-step on row pairs; the pair holding the band's last row first
#pragma unroll
        for (int ii = 0; ii < H2; ++ii) {
          const int i = (ii + H2 - 1) % H2;
          const f32x2 below = i + 1 < H2 ? Q1v[i + 1] : pk2(hi2(Q1v[0]), sQ1[(ty + 1) * BW + j]);
          const f32x2 left = pk2(sQ2r[i * L::QS], sQ2r[(i + H2) * L::QS]);
          const f32x2 right = pk2(sQ2r[i * L::QS + 1], sQ2r[(i + H2) * L::QS + 1]);
          const f32x2 d = sub2(add2(sub2(below, Q1v[i]), right), left);  // div_px
          const f32x2 fg = pk2(sFr[i * BW], sFr[(i + H2) * BW]);
          const f32x2 ub = fma2(SIG, d, U[i]);
          f32x2 un;
          if (FID == FID_L2) {
            un = fma2(UB, fg, mul2(UA, ub));
            if (MASK)
              un = pk2(((in_d >> i) & 1u) ? lo2(ub) : lo2(un), ((in_d >> (i + H2)) & 1u) ? hi2(ub) : hi2(un));
          } else {
            un = pk2(prox_ubar<FID>(lo2(ub), lo2(fg), MASK && ((in_d >> i) & 1u), c),
                     prox_ubar<FID>(hi2(ub), hi2(fg), MASK && ((in_d >> (i + H2)) & 1u), c));
          }
          U[i] = un;
          sUr[i * L::US] = lo2(un);
          sUr[(i + H2) * L::US] = hi2(un);
          if (ii == 0 && push_down) st_async_f32(remote_u, hi2(un), remote_mbU);
        }
        __syncthreads();
        if (need_uh) wait_u();  // u halo of iteration k
        // p-step on row pairs; the pair holding the band's first row first
#pragma unroll
        for (int i = 0; i < H2; ++i) {
          const f32x2 above = i > 0 ? U[i - 1] : pk2(sUr[-L::US], lo2(U[H2 - 1]));
          const f32x2 leftu = pk2(sUr[i * L::US - 1], sUr[(i + H2) * L::US - 1]);
          {
            const f32x2 tt = fma2(PC, sub2(U[i], above), fma2(PA, P1v[i], mul2(PB, H1v[i])));  // p_target
            const float l0 = i == 0 ? lim_top : 1.f;
            const f32x2 pn = pk2(fminf(fmaxf(lo2(tt), -l0), l0), fminf(fmaxf(hi2(tt), -1.f), 1.f));
            Q1v[i] = fma2(TH, sub2(pn, P1v[i]), pn);
            P1v[i] = pn;
          }
          {
            const f32x2 tt = fma2(PC, sub2(U[i], leftu), fma2(PA, P2v[i], mul2(PB, H2v[i])));
            const f32x2 pn = pk2(fminf(fmaxf(lo2(tt), -lim_left), lim_left),
                                 fminf(fmaxf(hi2(tt), -lim_left), lim_left));
            const f32x2 q2 = fma2(TH, sub2(pn, P2v[i]), pn);
            P2v[i] = pn;
            sQ2r[i * L::QS] = lo2(q2);
            sQ2r[(i + H2) * L::QS] = hi2(q2);
          }
          if (i == 0) {
            const float q10 = lo2(Q1v[0]);
            sQ1[ty * BW + j] = q10;
            if (push_up) st_async_f32(remote_q1, q10, remote_mbQ);
          }
        }
        if (last_row_here && s_bot) {
          float qB;
          p_update(pB, qB, -hi2(U[H2 - 1]), hB, c);
          sQ1[TR * BW + j] = qB;
        }
        if (right_lane) {
          const int lr = lr0 + j;
          float pr = sPR[lr], qr;
          p_update(pr, qr, -sU[(lr + 1) * L::US + 128], sHR[lr], c);
          sPR[lr] = pr;
          sQ2[lr * L::QS + 128] = qr;
        }
        __syncthreads();
      }
#pragma unroll
      for (int i = 0; i < H2; ++i) {
        u[i] = lo2(U[i]);
        u[i + H2] = hi2(U[i]);
        p1[i] = lo2(P1v[i]);
        p1[i + H2] = hi2(P1v[i]);
        p2[i] = lo2(P2v[i]);
        p2[i + H2] = hi2(P2v[i]);
      }
    } else {
      for (int k = 0; k < K; ++k) {
        Coef c;
        if (k < L::kMaxSmemCoef) {
          const float4 ca = *reinterpret_cast<const float4*>(sCo + 8 * k);
          const float4 cb = *reinterpret_cast<const float4*>(sCo + 8 * k + 4);
          c = Coef{ca.x, ca.y, ca.z, ca.w, cb.x, cb.y, cb.z, cb.w};
        } else {
          c = A.coef[k];
        }
        if (need_qh && k > 0) wait_q();  // pbar1 halo of iteration k-1
  #pragma unroll
        for (int rr = 0; rr < R; ++rr) {
          const int r = (rr + R - 1) % R;
          const float below = r + 1 < R ? q1[r + 1] : sQ1[(ty + 1) * BW + j];
          const float d = div_px(q1[r], below, sQ2r[r * L::QS], sQ2r[r * L::QS + 1]);
          u[r] = u_update<FID>(u[r], d, sFr[r * BW], MASK && ((in_d >> r) & 1u), c);
          sUr[r * L::US] = u[r];
          if (rr == 0 && push_down) st_async_f32(remote_u, u[R - 1], remote_mbU);
        }
        __syncthreads();
        if (need_uh) wait_u();  // u halo of iteration k
  #pragma unroll
        for (int r = 0; r < R; ++r) {
          const float above = r > 0 ? u[r - 1] : sUr[-L::US];
          p_update_lim(p1[r], q1[r], u[r] - above, h1[r], c, r == 0 ? lim_top : 1.f);
          float q2;
          p_update_lim(p2[r], q2, u[r] - sUr[r * L::US - 1], h2[r], c, lim_left);
          sQ2r[r * L::QS] = q2;
          if (r == 0) {
            sQ1[ty * BW + j] = q1[0];
            if (push_up) st_async_f32(remote_q1, q1[0], remote_mbQ);
          }
        }
        if (last_row_here && s_bot) {
          float qB;
          p_update(pB, qB, -u[R - 1], hB, c);
          sQ1[TR * BW + j] = qB;
        }
        if (right_lane) {
          const int lr = lr0 + j;
          float pr = sPR[lr], qr;
          p_update(pr, qr, -sU[(lr + 1) * L::US + 128], sHR[lr], c);
          sPR[lr] = pr;
          sQ2[lr * L::QS + 128] = qr;
        }
        __syncthreads();
      }
    }
    if (need_qh) wait_q();  // drain the last pbar1 halo (not read)

#pragma unroll
    for (int r = 0; r < R; ++r) {
      const int gi = r0 + i0 + r;
      A.u[(size_t)gi * g.W + gj] = u[r];
      A.P1[(size_t)(gi + a) * g.W + gj] = p1[r];
      A.P2[(size_t)gi * W2 + gj + b] = p2[r];
    }
    const Strips out = S.out(t);
    if (i0 == 0 && s_top) out.ST[(size_t)(a - 1) * g.W + gj] = p1[0];
    if (j == 0 && s_lft) {
#pragma unroll
      for (int r = 0; r < R; ++r) out.SL[(size_t)(b - 1) * g.H + r0 + i0 + r] = p2[r];
    }
    if (last_row_here && s_bot) {
      A.P1[(size_t)(r0 + 128 + a) * g.W + gj] = pB;
      out.SB[(size_t)a * g.W + gj] = pB;
    }
    if (right_lane) {
      const int gi = r0 + i0 + j;
      const float pr = sPR[lr0 + j];
      A.P2[(size_t)gi * W2 + c0 + 128 + b] = pr;
      out.SR[(size_t)b * g.H + gi] = pr;
    }
    };  // tile_body
    switch (S.fid(t)) {
      case FID_L2: tile_body(FidC<FID_L2>{}); break;
      case FID_L1: tile_body(FidC<FID_L1>{}); break;
      default: tile_body(FidC<FID_SEG>{}); break;
    }
  }
  cp_async_wait_all();
  cluster_arrive<true>();  // no CTA leaves while a neighbour may still write into it
  cluster_wait();
  if (timed_out) atomicOr(S.err(), 1);
}

template <int R, int TR, int CL, int MINB, int FID, bool MASK, bool PK>
__global__ void __launch_bounds__(128 * TR, MINB) k_fused_pa(const LocalArgs A) {
  fused_pa_body<R, TR, CL, FID, MASK, PK>(A, blockIdx.y, gridDim.y);
}

// Persistent kernel over the work list of a batch: cluster c runs tiles c, c + C, ...
// of the batch, each with its image's fidelity, parameters and coefficients.
template <int R, int TR, int CL, int MINB, bool PK>
__global__ void __launch_bounds__(128 * TR, MINB) k_fused_pa_batch(const BatchArgs B, int total) {
  fused_pa_run<R, TR, CL, false, PK>(BatchTiles{B, total}, blockIdx.y, gridDim.y);
}

struct Config {
  int BW, R, TR, CL;
  const char* name;
};

// Hardware mappings.  Class 0: tiles up to 32 x 32; class 1: up to 64 x 64; class 2:
// up to 128 x 128, where `variant` picks among the mappings (0 is the default).
constexpr Config kConfigs[] = {
    {32, 8, 4, 1, "bw32_r8_tr4_cl1"},      // class 0
    {64, 8, 8, 1, "bw64_r8_tr8_cl1"},      // class 1
    {128, 8, 2, 8, "bw128_r8_tr2_cl8"},    // class 2, variant 0: 256 threads, 2 CTAs/SM
    {128, 8, 4, 4, "bw128_r8_tr4_cl4"},    // class 2, variant 1: 512 threads, 1 CTA/SM
    {128, 16, 2, 4, "bw128_r16_tr2_cl4"},  // class 2, variant 2: 256 threads, 16 rows/thread
};
constexpr int kNumVariants = 16;

template <int BW, int R, int TR, int CL, int FID, bool MASK, bool ADAPT>
cudaError_t launch_one(const LocalArgs& a, cudaStream_t st) {
  using L = SmemLayout<BW, R, TR>;
  // configurations above 48 KB of shared memory need the opt-in attribute, set by
  // fused_prepare() when the handle is created (never during graph capture)
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(CL, a.g.NC, a.g.NR);
  cfg.blockDim = dim3(BW, TR, 1);
  cfg.dynamicSmemBytes = L::BYTES;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = CL;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k_fused<BW, R, TR, CL, FID, MASK, ADAPT>, a);
}

template <int BW, int R, int TR, int CL, bool ADAPT>
cudaError_t launch_fid_a(const LocalArgs& a, int fid, cudaStream_t st) {
  const bool m = a.mask != nullptr;
  switch (fid) {
    case FID_L2:
      return m ? launch_one<BW, R, TR, CL, FID_L2, true, ADAPT>(a, st)
               : launch_one<BW, R, TR, CL, FID_L2, false, ADAPT>(a, st);
    case FID_L1:
      return m ? launch_one<BW, R, TR, CL, FID_L1, true, ADAPT>(a, st)
               : launch_one<BW, R, TR, CL, FID_L1, false, ADAPT>(a, st);
    default: return launch_one<BW, R, TR, CL, FID_SEG, false, ADAPT>(a, st);
  }
}

template <int BW, int R, int TR, int CL>
cudaError_t launch_fid(const LocalArgs& a, int fid, cudaStream_t st) {
  return a.inner_tol2 > 0.0 ? launch_fid_a<BW, R, TR, CL, true>(a, fid, st)
                            : launch_fid_a<BW, R, TR, CL, false>(a, fid, st);
}

template <int R, int TR, int CL, int MINB, int FID, bool MASK>
cudaError_t launch_full_one(const LocalArgs& a, cudaStream_t st) {
  using L = FullLayout<R, TR>;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(CL, a.g.NC, a.g.NR);
  cfg.blockDim = dim3(128, TR, 1);
  cfg.dynamicSmemBytes = L::BYTES;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = CL;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k_fused_full<R, TR, CL, MINB, FID, MASK>, a);
}

template <int R, int TR, int CL, int MINB>
cudaError_t launch_full(const LocalArgs& a, int fid, cudaStream_t st) {
  const bool m = a.mask != nullptr;
  switch (fid) {
    case FID_L2: return m ? launch_full_one<R, TR, CL, MINB, FID_L2, true>(a, st) : launch_full_one<R, TR, CL, MINB, FID_L2, false>(a, st);
    case FID_L1: return m ? launch_full_one<R, TR, CL, MINB, FID_L1, true>(a, st) : launch_full_one<R, TR, CL, MINB, FID_L1, false>(a, st);
    default: return launch_full_one<R, TR, CL, MINB, FID_SEG, false>(a, st);
  }
}

template <int R, int TR, int CL, int MINB, int FID, bool MASK>
cudaError_t launch_async_one(const LocalArgs& a, cudaStream_t st) {
  using AL = AsyncLayout<R, TR>;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(CL, a.g.NC, a.g.NR);
  cfg.blockDim = dim3(128, TR, 1);
  cfg.dynamicSmemBytes = AL::BYTES;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = CL;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k_fused_async<R, TR, CL, MINB, FID, MASK>, a);
}

template <int R, int TR, int CL, int MINB>
cudaError_t launch_async(const LocalArgs& a, int fid, cudaStream_t st) {
  const bool m = a.mask != nullptr;
  switch (fid) {
    case FID_L2: return m ? launch_async_one<R, TR, CL, MINB, FID_L2, true>(a, st) : launch_async_one<R, TR, CL, MINB, FID_L2, false>(a, st);
    case FID_L1: return m ? launch_async_one<R, TR, CL, MINB, FID_L1, true>(a, st) : launch_async_one<R, TR, CL, MINB, FID_L1, false>(a, st);
    default: return launch_async_one<R, TR, CL, MINB, FID_SEG, false>(a, st);
  }
}

template <int R, int TR, int CL, int MINB>
cudaError_t launch_async_batch(const BatchArgs& B, int total_tiles, cudaStream_t st) {
  using AL = AsyncLayout<R, TR>;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(CL, total_tiles, 1);
  cfg.blockDim = dim3(128, TR, 1);
  cfg.dynamicSmemBytes = AL::BYTES;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = CL;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k_fused_async_batch<R, TR, CL, MINB>, B);
}

// clusters of the persistent kernel resident at once, per device and instantiation
template <int R, int TR, int CL, int MINB, int FID, bool MASK, bool PK>
int& pa_clusters(int dev) {
  static int n[64] = {0};
  return n[dev & 63];
}

template <int R, int TR, int CL, int MINB, int FID, bool MASK, bool PK>
cudaError_t launch_pa_one(const LocalArgs& a, cudaStream_t st) {
  using P = PaLayout<R, TR>;
  int dev = 0;
  cudaGetDevice(&dev);
  const int tiles = a.g.NR * a.g.NC;
  int nc = pa_clusters<R, TR, CL, MINB, FID, MASK, PK>(dev);
  if (nc <= 0 || nc > tiles) nc = tiles;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(CL, nc, 1);
  cfg.blockDim = dim3(128, TR, 1);
  cfg.dynamicSmemBytes = P::BYTES;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = CL;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k_fused_pa<R, TR, CL, MINB, FID, MASK, PK>, a);
}

template <int R, int TR, int CL, int MINB, bool PK>
cudaError_t launch_pa(const LocalArgs& a, int fid, cudaStream_t st) {
  const bool m = a.mask != nullptr;
  switch (fid) {
    case FID_L2: return m ? launch_pa_one<R, TR, CL, MINB, FID_L2, true, PK>(a, st) : launch_pa_one<R, TR, CL, MINB, FID_L2, false, PK>(a, st);
    case FID_L1: return m ? launch_pa_one<R, TR, CL, MINB, FID_L1, true, PK>(a, st) : launch_pa_one<R, TR, CL, MINB, FID_L1, false, PK>(a, st);
    default: return launch_pa_one<R, TR, CL, MINB, FID_SEG, false, PK>(a, st);
  }
}

// shared-memory opt-in, and how many clusters fit at once (0 disables persistence)
template <int R, int TR, int CL, int MINB, int FID, bool MASK, bool PK>
cudaError_t prepare_pa_one() {
  using P = PaLayout<R, TR>;
  auto kern = k_fused_pa<R, TR, CL, MINB, FID, MASK, PK>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)P::BYTES);
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(CL, 1024, 1);
  cfg.blockDim = dim3(128, TR, 1);
  cfg.dynamicSmemBytes = P::BYTES;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = CL;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  int n = 0;
  if (cudaOccupancyMaxActiveClusters(&n, kern, &cfg) != cudaSuccess) {
    cudaGetLastError();
    n = 0;
  }
  int dev = 0;
  cudaGetDevice(&dev);
  pa_clusters<R, TR, CL, MINB, FID, MASK, PK>(dev) = n;
  return cudaSuccess;
}

template <int R, int TR, int CL, int MINB, bool PK>
cudaError_t prepare_pa() {
  cudaError_t e;
  if ((e = prepare_pa_one<R, TR, CL, MINB, FID_L2, false, PK>()) != cudaSuccess) return e;
  if ((e = prepare_pa_one<R, TR, CL, MINB, FID_L2, true, PK>()) != cudaSuccess) return e;
  if ((e = prepare_pa_one<R, TR, CL, MINB, FID_L1, false, PK>()) != cudaSuccess) return e;
  if ((e = prepare_pa_one<R, TR, CL, MINB, FID_L1, true, PK>()) != cudaSuccess) return e;
  return prepare_pa_one<R, TR, CL, MINB, FID_SEG, false, PK>();
}

// persistent batch kernel: clusters resident at once (per device), launch
template <int R, int TR, int CL, int MINB, bool PK>
int& pa_batch_clusters(int dev) {
  static int n[64] = {0};
  return n[dev & 63];
}

template <int R, int TR, int CL, int MINB, bool PK>
cudaError_t prepare_pa_batch() {
  using P = PaLayout<R, TR>;
  auto kern = k_fused_pa_batch<R, TR, CL, MINB, PK>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)P::BYTES);
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(CL, 1024, 1);
  cfg.blockDim = dim3(128, TR, 1);
  cfg.dynamicSmemBytes = P::BYTES;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = CL;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  int n = 0;
  if (cudaOccupancyMaxActiveClusters(&n, kern, &cfg) != cudaSuccess) {
    cudaGetLastError();
    n = 0;
  }
  int dev = 0;
  cudaGetDevice(&dev);
  pa_batch_clusters<R, TR, CL, MINB, PK>(dev) = n;
  return cudaSuccess;
}

template <int R, int TR, int CL, int MINB, bool PK>
cudaError_t launch_pa_batch(const BatchArgs& B, int total_tiles, cudaStream_t st) {
  using P = PaLayout<R, TR>;
  int dev = 0;
  cudaGetDevice(&dev);
  int nc = pa_batch_clusters<R, TR, CL, MINB, PK>(dev);
  if (nc <= 0 || nc > total_tiles) nc = total_tiles;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(CL, nc, 1);
  cfg.blockDim = dim3(128, TR, 1);
  cfg.dynamicSmemBytes = P::BYTES;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = CL;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k_fused_pa_batch<R, TR, CL, MINB, PK>, B, total_tiles);
}

template <int R, int TR, int CL, int MINB, int FID, bool MASK>
cudaError_t prepare_async_one() {
  using AL = AsyncLayout<R, TR>;
  return cudaFuncSetAttribute(k_fused_async<R, TR, CL, MINB, FID, MASK>,
                              cudaFuncAttributeMaxDynamicSharedMemorySize, (int)AL::BYTES);
}

template <int R, int TR, int CL, int MINB>
cudaError_t prepare_async() {
  cudaError_t e;
  if ((e = prepare_async_one<R, TR, CL, MINB, FID_L2, false>()) != cudaSuccess) return e;
  if ((e = prepare_async_one<R, TR, CL, MINB, FID_L2, true>()) != cudaSuccess) return e;
  if ((e = prepare_async_one<R, TR, CL, MINB, FID_L1, false>()) != cudaSuccess) return e;
  if ((e = prepare_async_one<R, TR, CL, MINB, FID_L1, true>()) != cudaSuccess) return e;
  return prepare_async_one<R, TR, CL, MINB, FID_SEG, false>();
}

template <int R, int NW, int CL, int MINB, int FID, bool MASK>
cudaError_t launch_wr_one(const LocalArgs& a, cudaStream_t st) {
  using L = WrLayout<R, NW>;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(CL, a.g.NC, a.g.NR);
  cfg.blockDim = dim3(32 * NW, 1, 1);
  cfg.dynamicSmemBytes = L::BYTES;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = CL;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k_fused_wr<R, NW, CL, MINB, FID, MASK>, a);
}

template <int R, int NW, int CL, int MINB>
cudaError_t launch_wr(const LocalArgs& a, int fid, cudaStream_t st) {
  const bool m = a.mask != nullptr;
  switch (fid) {
    case FID_L2: return m ? launch_wr_one<R, NW, CL, MINB, FID_L2, true>(a, st) : launch_wr_one<R, NW, CL, MINB, FID_L2, false>(a, st);
    case FID_L1: return m ? launch_wr_one<R, NW, CL, MINB, FID_L1, true>(a, st) : launch_wr_one<R, NW, CL, MINB, FID_L1, false>(a, st);
    default: return launch_wr_one<R, NW, CL, MINB, FID_SEG, false>(a, st);
  }
}

template <int R, int TR, int CL, int MINB, int FID, bool MASK>
cudaError_t prepare_full_one() {
  using L = FullLayout<R, TR>;
  return cudaFuncSetAttribute(k_fused_full<R, TR, CL, MINB, FID, MASK>,
                              cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L::BYTES);
}

template <int R, int TR, int CL, int MINB>
cudaError_t prepare_full() {
  cudaError_t e;
  if ((e = prepare_full_one<R, TR, CL, MINB, FID_L2, false>()) != cudaSuccess) return e;
  if ((e = prepare_full_one<R, TR, CL, MINB, FID_L2, true>()) != cudaSuccess) return e;
  if ((e = prepare_full_one<R, TR, CL, MINB, FID_L1, false>()) != cudaSuccess) return e;
  if ((e = prepare_full_one<R, TR, CL, MINB, FID_L1, true>()) != cudaSuccess) return e;
  return prepare_full_one<R, TR, CL, MINB, FID_SEG, false>();
}

template <int BW, int R, int TR, int CL, int FID, bool MASK>
cudaError_t prepare_one() {
  using L = SmemLayout<BW, R, TR>;
  cudaError_t e = cudaFuncSetAttribute(k_fused<BW, R, TR, CL, FID, MASK, false>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L::BYTES);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(k_fused<BW, R, TR, CL, FID, MASK, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)L::BYTES);
}

template <int BW, int R, int TR, int CL>
cudaError_t prepare_fid() {
  cudaError_t e;
  if ((e = prepare_one<BW, R, TR, CL, FID_L2, false>()) != cudaSuccess) return e;
  if ((e = prepare_one<BW, R, TR, CL, FID_L2, true>()) != cudaSuccess) return e;
  if ((e = prepare_one<BW, R, TR, CL, FID_L1, false>()) != cudaSuccess) return e;
  if ((e = prepare_one<BW, R, TR, CL, FID_L1, true>()) != cudaSuccess) return e;
  return prepare_one<BW, R, TR, CL, FID_SEG, false>();
}

// index into kConfigs for a tile shape and variant, -1 if none fits
int pick(int mr, int mc, int variant) {
  if (mc <= 32 && mr <= 32) return 0;
  if (mc <= 64 && mr <= 64) return 1;
  if (mc <= 128 && mr <= 128 && variant >= 0 && variant < kNumVariants) return 2 + (variant < 3 ? variant : 0);
  return -1;
}

}  // namespace

void fused_max_tile(int* rows, int* cols) {
  *rows = 128;
  *cols = 128;
}

int fused_num_variants() { return kNumVariants; }

const char* fused_config_name(int mr, int mc, int variant) {
  const int q = pick(mr, mc, variant);
  return q < 0 ? "none" : kConfigs[q].name;
}

cudaError_t fused_prepare() {
  cudaError_t e;
  if ((e = prepare_fid<32, 8, 4, 1>()) != cudaSuccess) return e;
  if ((e = prepare_fid<64, 8, 8, 1>()) != cudaSuccess) return e;
  if ((e = prepare_fid<128, 8, 2, 8>()) != cudaSuccess) return e;
  if ((e = prepare_fid<128, 8, 4, 4>()) != cudaSuccess) return e;
  if ((e = prepare_fid<128, 16, 2, 4>()) != cudaSuccess) return e;
  if ((e = prepare_full<8, 4, 4, 1>()) != cudaSuccess) return e;
  if ((e = prepare_async<8, 2, 8, 2>()) != cudaSuccess) return e;
  if ((e = prepare_async<8, 4, 4, 1>()) != cudaSuccess) return e;
  if ((e = prepare_pa<8, 2, 8, 2, true>()) != cudaSuccess) return e;
  if ((e = prepare_pa<8, 2, 8, 2, false>()) != cudaSuccess) return e;
  if ((e = prepare_pa<8, 4, 4, 1, false>()) != cudaSuccess) return e;
  if ((e = prepare_pa<4, 4, 8, 2, true>()) != cudaSuccess) return e;
  if ((e = prepare_pa<16, 1, 8, 2, true>()) != cudaSuccess) return e;
  if ((e = prepare_pa<8, 2, 8, 3, true>()) != cudaSuccess) return e;
  if ((e = prepare_pa_batch<8, 2, 8, 2, true>()) != cudaSuccess) return e;
  if ((e = fused_pg_prepare()) != cudaSuccess) return e;
  if ((e = fused_mt_prepare()) != cudaSuccess) return e;
  if ((e = fused_wrow_prepare()) != cudaSuccess) return e;
  if ((e = fused_ps_prepare()) != cudaSuccess) return e;
  if ((e = fused_mt4_prepare()) != cudaSuccess) return e;
  if ((e = cudaFuncSetAttribute(k_fused_async_batch<8, 2, 8, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)AsyncLayout<8, 2>::BYTES)) != cudaSuccess)
    return e;
  return cudaFuncSetAttribute(k_fused_async_batch<8, 4, 4, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)AsyncLayout<8, 4>::BYTES);
}

cudaError_t launch_fused_batch(const BatchArgs& B, int total_tiles, int variant, cudaStream_t st) {
  if (variant == 1) return launch_async_batch<8, 2, 8, 2>(B, total_tiles, st);
  if (variant == 2) return launch_async_batch<8, 4, 4, 1>(B, total_tiles, st);
  if (variant == 3) return launch_pa_batch<8, 2, 8, 2, true>(B, total_tiles, st);
  return launch_fused_mt_batch(B, total_tiles, st);
}

cudaError_t launch_fused_local(const LocalArgs& a, int fid, int variant, cudaStream_t st) {
  // largest tile of the (ragged) partition
  const int mr = (a.g.H + a.g.NR - 1) / a.g.NR, mc = (a.g.W + a.g.NC - 1) / a.g.NC;
  if (a.inner_tol2 > 0.0) variant = 0;  // adaptive stopping: the cluster-barrier kernel only
  if (a.inner_tol2 <= 0.0 && a.g.H == 128 * a.g.NR && a.g.W == 128 * a.g.NC) {  // every tile exactly 128 x 128
    switch (variant) {
      case 0:  // default: persistent, 4 x 4 micro-tiles, one warp per thread row, 3 CTAs per SM, tensor copies
        if (fused_mt4_supported(a)) return launch_fused_mt4(a, fid, true, st);
        return fused_mt_supported(a) ? launch_fused_mt(a, fid, st) : launch_pa<8, 2, 8, 2, true>(a, fid, st);
      case 1: return launch_async<8, 2, 8, 2>(a, fid, st);      // async halos, one subdomain per cluster
      case 2: return launch_full<8, 4, 4, 1>(a, fid, st);       // cluster barrier per half-step: 512 threads
      case 3: return launch_wr<2, 8, 8, 2>(a, fid, st);         // warp rows, per-warp mbarriers
      case 4: return launch_pa<8, 4, 4, 1, false>(a, fid, st);  // persistent, async halos, prefetch: 512 threads
      case 5: return launch_async<8, 4, 4, 1>(a, fid, st);      // async halos: 512 threads
      case 6: return launch_pa<8, 2, 8, 2, false>(a, fid, st);  // variant 11 with scalar arithmetic
      case 7: return launch_pa<4, 4, 8, 2, true>(a, fid, st);   // variant 11 with 4 rows per thread: 512 threads
      case 8: return launch_pa<16, 1, 8, 2, true>(a, fid, st);  // variant 11 with 16 rows per thread: 128 threads
      case 9: return launch_pa<8, 2, 8, 3, true>(a, fid, st);   // variant 11 at 3 CTAs per SM (80 registers)
      case 10: return launch_fused_pg(a, fid, st);              // one halo exchange per inner iteration
      case 11: return launch_pa<8, 2, 8, 2, true>(a, fid, st);  // persistent column mapping, packed pairs
      case 12:                                                  // warp per row pair, named barriers, bulk copies
        return fused_wrow_supported(a) ? launch_fused_wrow(a, fid, st) : launch_pa<8, 2, 8, 2, true>(a, fid, st);
      case 13:                                                  // variant 11 with 16-byte copies, out-buffer
        return fused_ps_supported(a) ? launch_fused_ps(a, fid, st) : launch_pa<8, 2, 8, 2, true>(a, fid, st);
      case 14:                                                  // 2 x 4 micro-tiles, 256 threads, 2 CTAs per SM
        return fused_mt_supported(a) ? launch_fused_mt(a, fid, st) : launch_pa<8, 2, 8, 2, true>(a, fid, st);
      case 15:                                                  // variant 0 moving the state with cp.async
        return fused_mt4_supported(a) ? launch_fused_mt4(a, fid, false, st) : launch_pa<8, 2, 8, 2, true>(a, fid, st);
      default: return cudaErrorInvalidValue;
    }
  }
  switch (pick(mr, mc, variant)) {
    case 0: return launch_fid<32, 8, 4, 1>(a, fid, st);
    case 1: return launch_fid<64, 8, 8, 1>(a, fid, st);
    case 2: return launch_fid<128, 8, 2, 8>(a, fid, st);
    case 3: return launch_fid<128, 8, 4, 4>(a, fid, st);
    case 4: return launch_fid<128, 16, 2, 4>(a, fid, st);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace ddtv
