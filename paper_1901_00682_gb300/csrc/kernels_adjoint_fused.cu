// Tile-fused reverse pass of one outer iteration's local solves.
//
// One launch recomputes the K inner iterations of every subdomain (the fused forward
// kernel's arithmetic, bit for bit) while recording the tape in shared memory (ubar_k
// of every pixel and the projection's pass bits of every dof), then runs the K
// reverse iterations of kernels_adjoint.cu (same formulas, same operation order) with
// the adjoint state in registers.  Global memory is touched once per outer iteration
// (load the state, the proximal centre, the adjoint of u and p; store the adjoint of u
// and p, the adjoint of the proximal centre on the subdomain's sides, and add to the
// adjoint of f), instead of streaming every field through HBM at every inner step.
//
// Mapping (as k_fused): a subdomain of mr x mc pixels is owned by a cluster of CL
// CTAs; CTA `rank` owns TR*R rows, thread (j, ty) owns column j and R consecutive
// rows.  The reverse iteration has the forward's communication pattern: the u-step's
// adjoint (Ad, the adjoint of the divergence) is needed by the row below and the
// column to the right, the p-step's adjoint (a_t of every dof) by the row above and the
// column to the left; halo rows cross CTAs through DSMEM stores ordered by the split
// cluster barrier, as in the forward kernel.
#include "fused_common.cuh"
#include "internal.cuh"

namespace ddtv {

namespace {

__device__ __forceinline__ uint32_t s_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint32_t to_rank(uint32_t addr, int rank) {
  uint32_t out;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(out) : "r"(addr), "r"(rank));
  return out;
}

__device__ __forceinline__ void st_remote(uint32_t addr, float v) {
  asm volatile("st.shared::cluster.f32 [%0], %1;" ::"r"(addr), "f"(v) : "memory");
}

template <bool RELEASE>
__device__ __forceinline__ void cl_arrive() {
  if (RELEASE)
    asm volatile("barrier.cluster.arrive.release.aligned;" ::: "memory");
  else
    asm volatile("barrier.cluster.arrive.relaxed.aligned;" ::: "memory");
}

__device__ __forceinline__ void cl_wait() { asm volatile("barrier.cluster.wait.acquire.aligned;" ::: "memory"); }

// p-step with the clamp to [-lim, lim] (lim = 0 pins an inactive dof at 0), as the
// fused forward kernel; returns the projection's pass bit (0 for an inactive dof).
__device__ __forceinline__ uint32_t p_step_bit(float& p, float& pbar, float du, float phat, const Coef& c, float lim) {
  const float t = p_target(p, du, phat, c);
  const float pn = clamp_abs(t, lim);
  pbar = fmaf(c.th, pn - p, pn);
  p = pn;
  return (lim > 0.f && t >= -1.0f && t <= 1.0f) ? 1u : 0u;
}

// du'/dubar, du'/df, du'/dalpha of u' = prox(ubar) (Section 3 proximity maps); fg is f
// (L2, L1) or g = (f - c1)^2 - (f - c2)^2 (SEG), as in the forward's shared array.
template <int FID>
__device__ __forceinline__ void prox_partials_fg(float ub, float fg, bool in_d, float c1, float c2, const Coef& c,
                                                 float& dub, float& df, float& dal) {
  if (FID == FID_SEG) {
    const float x = fmaf(-c.s, fg, ub);
    const bool pass = x >= 0.0f && x <= 1.0f;
    dub = pass ? 1.0f : 0.0f;
    dal = pass ? -c.sig * fg : 0.0f;
    df = pass ? -c.s * (2.0f * (c2 - c1)) : 0.0f;
    return;
  }
  if (in_d) {
    dub = 1.0f;
    df = 0.0f;
    dal = 0.0f;
    return;
  }
  if (FID == FID_L2) {
    dub = c.ua;
    df = c.ub;
    dal = c.sig * c.ua * c.ua * (fg - ub);
    return;
  }
  const float v = ub - fg;
  const bool pass = fabsf(v) - c.s > 0.0f;
  dub = pass ? 1.0f : 0.0f;
  df = pass ? 0.0f : 1.0f;
  dal = pass ? (v > 0.0f ? -c.sig : c.sig) : 0.0f;
}

// One dof of the reverse p-step (the formulas of kernels_adjoint.cu adj_dof).
__device__ __forceinline__ void adj_dof_reg(float& AP, float& AQ, float& APh, bool pass, float aq_new, const Coef& c,
                                            float opq, bool first, bool last) {
  const float aq = AQ;
  const float at = pass ? AP + opq * aq : 0.0f;
  const float aph = (first ? 0.0f : APh) + c.pb * at;
  const float ap = c.pa * at - c.th * aq;
  APh = aph;
  if (last) {
    AP = (ap + aq_new) + aph;
    AQ = 0.0f;
  } else {
    AP = ap;
    AQ = aq_new;
  }
}

template <int BW, int R, int TR>
struct AdjLayout {
  static constexpr int BAND = TR * R;
  static constexpr int NT = BW * TR;
  static constexpr int US = BW + 1;                 // u / Ad rows; index 0 = zero pad left of column 0
  static constexpr int QS = BW + 1;                 // pbar2 / a_t2 rows; index mc = the right side
  static constexpr int U = 0;                       // BAND x US
  static constexpr int UH = U + BAND * US;          // US: row above the band (CTA above's last row)
  static constexpr int Q2 = UH + US;                // BAND x QS
  static constexpr int Q1 = Q2 + BAND * QS;         // TR x BW: first row of every thread row
  static constexpr int Q1H = Q1 + TR * BW;          // BW: row below the band (CTA below's first row)
  static constexpr int F = Q1H + BW;                // BAND x BW: f (or g)
  static constexpr int PR = F + BAND * BW;          // BAND: right-side p / its adjoint AP
  static constexpr int HR = PR + BAND;              // BAND: right-side phat / its adjoint AQ
  static constexpr int XR = HR + BAND;              // BAND: right-side adjoint of phat
  static constexpr int FLOATS = XR + BAND;
  static constexpr size_t BYTES = sizeof(float) * FLOATS;
  // tape of one CTA in global memory: K x R x NT ubar, then K x NT pass-bit words
  static constexpr size_t tape_floats(int K) { return (size_t)K * (R + 1) * NT; }
};

// Pass-bit word of one thread and iteration: bit r = p1 dof of band row r, bit 8 + r =
// p2 dof of row r, bit 16 = the tile's bottom side, bit 17 + r = right side of row r.
// The tape lives in global memory, one contiguous slice per CTA (Z.tape); it is
// written and read back within the same launch, so it stays in L2.
template <int BW, int R, int TR, int CL, int MINB, int FID, bool MASK>
__global__ void __launch_bounds__(BW* TR, MINB) k_adj_fused(const LocalArgs A, const AdjArgs Z) {
  static_assert(R <= 8, "pass-bit word layout");
  using L = AdjLayout<BW, R, TR>;
  constexpr int BAND = L::BAND, NT = L::NT;
  extern __shared__ __align__(16) float smem[];
  float* sU = smem + L::U;
  float* sUh = smem + L::UH;
  float* sQ2 = smem + L::Q2;
  float* sQ1 = smem + L::Q1;
  float* sQ1h = smem + L::Q1H;
  float* sF = smem + L::F;
  float* sPR = smem + L::PR;
  float* sHR = smem + L::HR;
  float* sXR = smem + L::XR;
  const int K = A.K;
  const Grid g = A.g;
  const int rank = CL > 1 ? (int)blockIdx.x : 0;
  const int b = blockIdx.y, a = blockIdx.z;
  float* tapeU = Z.tape + ((size_t)(a * g.NC + b) * CL + rank) * L::tape_floats(K);
  uint32_t* tapeM = reinterpret_cast<uint32_t*>(tapeU + (size_t)K * R * NT);
  const int r0 = part_start(a, g.H, g.NR), mr = part_start(a + 1, g.H, g.NR) - r0;
  const int c0 = part_start(b, g.W, g.NC), mc = part_start(b + 1, g.W, g.NC) - c0;
  const bool s_top = a > 0, s_bot = a + 1 < g.NR, s_lft = b > 0, s_rgt = b + 1 < g.NC;
  const int j = threadIdx.x, ty = threadIdx.y, tid = ty * BW + j;
  const int lr0 = ty * R;
  const int i0 = rank * BAND + lr0;
  const bool col_ok = j < mc;
  const int W2 = g.W + g.NC;
  const int gj = c0 + j;
  const float tau = A.tau;
  const float lim_left = (j == 0 && !s_lft) ? 0.f : 1.f;
  const float lim_top = (i0 == 0 && !s_top) ? 0.f : 1.f;
  const int rb = mr - 1 - i0;  // r of the tile's last row, if in [0, R)
  const bool right_thr = j == mc - 1 && s_rgt;
  const bool push_down = CL > 1 && ty == TR - 1 && rank + 1 < CL;
  const bool push_up = CL > 1 && ty == 0 && rank > 0;
  uint32_t remote_uh = 0, remote_q1h = 0;
  if (push_down) remote_uh = to_rank(s_addr(sUh + 1 + j), rank + 1);
  if (push_up) remote_q1h = to_rank(s_addr(sQ1h + j), rank - 1);

  float u[R], p1[R], p2[R], h1[R], h2[R], q1[R];
  uint32_t in_d = 0;
  float pB = 0.f, hB = 0.f, qB = 0.f;

  // ---- load the tile's state and build the proximal centre (as k_fused)
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
    sU[(lr0 + r) * L::US] = 0.f;
    if (col_ok) sQ2[(lr0 + r) * L::QS + j] = a2;
  }
  qB = pB;
  sQ1[ty * BW + j] = q1[0];
  if (push_up) st_remote(remote_q1h, q1[0]);
  __syncthreads();
  if (CL > 1) {
    if (push_up) cl_arrive<true>(); else cl_arrive<false>();
  }

  // ---- forward: K inner iterations, recording the tape
  for (int k = 0; k < K; ++k) {
    const Coef c = A.coef[k];
    float* tU = tapeU + (size_t)k * R * NT;
    uint32_t bits = 0;
    auto u_px = [&](int r) {
      const int lr = lr0 + r;
      float below;
      if (r == rb) below = qB;
      else if (r + 1 < R) below = q1[r + 1];
      else if (ty + 1 < TR) below = sQ1[(ty + 1) * BW + j];
      else below = sQ1h[j];
      const float d = div_px(q1[r], below, sQ2[lr * L::QS + j], sQ2[lr * L::QS + j + 1]);
      const float ub = fmaf(c.sig, d, u[r]);
      tU[r * NT + tid] = ub;
      u[r] = prox_ubar<FID>(ub, sF[lr * BW + j], MASK && ((in_d >> r) & 1u), c);
      sU[lr * L::US + j + 1] = u[r];
    };
    auto p_px = [&](int r) {
      const int lr = lr0 + r;
      float above;
      if (r > 0) above = u[r - 1];
      else if (ty > 0) above = sU[(lr - 1) * L::US + j + 1];
      else above = sUh[j + 1];
      bits |= p_step_bit(p1[r], q1[r], u[r] - above, h1[r], c, r == 0 ? lim_top : 1.f) << r;
      float q2;
      bits |= p_step_bit(p2[r], q2, u[r] - sU[lr * L::US + j], h2[r], c, lim_left) << (8 + r);
      if (r == rb && s_bot) bits |= p_step_bit(pB, qB, -u[r], hB, c, 1.f) << 16;
      if (right_thr) {
        float pr = sPR[lr], qr;
        bits |= p_step_bit(pr, qr, -u[r], sHR[lr], c, 1.f) << (17 + r);
        sPR[lr] = pr;
        sQ2[lr * L::QS + mc] = qr;
      }
      if (col_ok) sQ2[lr * L::QS + j] = q2;
    };
    if (CL > 1) cl_wait();
    u_px(R - 1);
    if (push_down) st_remote(remote_uh, u[R - 1]);
    if (CL > 1) {
      if (push_down) cl_arrive<true>(); else cl_arrive<false>();
    }
#pragma unroll
    for (int r = 0; r + 1 < R; ++r) u_px(r);
    __syncthreads();
    if (CL > 1) cl_wait();
    p_px(0);
    sQ1[ty * BW + j] = q1[0];
    if (push_up) st_remote(remote_q1h, q1[0]);
    if (CL > 1) {
      if (push_up) cl_arrive<true>(); else cl_arrive<false>();
    }
#pragma unroll
    for (int r = 1; r < R; ++r) p_px(r);
    tapeM[(size_t)k * NT + tid] = bits;
    __syncthreads();
  }
  if (CL > 1) cl_wait();  // every forward halo has landed; the shared arrays are reused below

  // ---- reverse.  Registers: adjoints of u, p1, p2, pbar1 (AQ1), pbar2 (AQ2), phat1,
  // phat2 and of the bottom side; the right side's (AP, AQ, APhat) live in sPR, sHR,
  // sXR.  Shared arrays: sU = Ad (sUh: the CTA above's last row, 0 above the tile),
  // sQ2 = a_t of the p2 dofs (column mc: right side), sQ1 / sQ1h = a_t of the first p1
  // row of every thread row / of the band below.
  float Au[R], AP1[R], AP2[R], AQ1[R], AQ2[R], AH1[R], AH2[R], Afr[R];
  float APB = 0.f, AQB = 0.f, AHB = 0.f, atB = 0.f;
  // the thread's share of dL/dalpha: compensated float32 sum (Kahan), float64 across
  // threads (a float64 add per pixel and iteration keeps the slow float64 pipe busy)
  float acc_s = 0.f, acc_c = 0.f;
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const int i = i0 + r;
    float au = 0.f, ap1 = 0.f, ap2 = 0.f;
    if (col_ok && i < mr) {
      const int gi = r0 + i;
      au = Z.Au[(size_t)gi * g.W + gj];
      ap1 = Z.AP1[(size_t)(gi + a) * g.W + gj];
      ap2 = Z.AP2[(size_t)gi * W2 + gj + b];
      if (i == mr - 1 && s_bot) APB = Z.AP1[(size_t)(gi + a + 1) * g.W + gj];
      if (right_thr) {
        sPR[lr0 + r] = Z.AP2[(size_t)gi * W2 + gj + b + 1];
        sHR[lr0 + r] = 0.f;
      }
    }
    Au[r] = au;
    AP1[r] = ap1;
    AP2[r] = ap2;
    AQ1[r] = 0.f;
    AQ2[r] = 0.f;
    AH1[r] = 0.f;
    AH2[r] = 0.f;
    Afr[r] = 0.f;
  }
  // a_t of iteration k (pass bits and theta of k) from the current AP, AQ: exchanged
  auto publish_at = [&](int k, bool row0_only) {
    const Coef c = A.coef[k];
    const float opq = 1.0f + c.th;
    const uint32_t bits = tapeM[(size_t)k * NT + tid];
#pragma unroll
    for (int r = 0; r < R; ++r) {
      if (row0_only && r > 0) break;
      const int lr = lr0 + r;
      const float at2 = ((bits >> (8 + r)) & 1u) ? AP2[r] + opq * AQ2[r] : 0.0f;
      if (col_ok) sQ2[lr * L::QS + j] = at2;
      if (right_thr) sQ2[lr * L::QS + mc] = ((bits >> (17 + r)) & 1u) ? sPR[lr] + opq * sHR[lr] : 0.0f;
    }
    const float at10 = (bits & 1u) ? AP1[0] + opq * AQ1[0] : 0.0f;
    sQ1[ty * BW + j] = at10;
    if (push_up) st_remote(remote_q1h, at10);
    if (rb >= 0 && rb < R) atB = (s_bot && ((bits >> 16) & 1u)) ? APB + opq * AQB : 0.0f;
  };
  if (j == mc - 1 && !s_rgt) {
    for (int r = 0; r < R; ++r) sQ2[(lr0 + r) * L::QS + mc] = 0.f;  // no right side: a_t = 0
  }
  publish_at(K - 1, false);
  __syncthreads();
  if (CL > 1) {
    if (push_up) cl_arrive<true>(); else cl_arrive<false>();
  }

  for (int k = K - 1; k >= 0; --k) {
    const Coef c = A.coef[k];
    const float opq = 1.0f + c.th;
    const uint32_t bits = tapeM[(size_t)k * NT + tid];
    const float* tU = tapeU + (size_t)k * R * NT;
    float ubk[R];  // this iteration's tape, loaded before the barrier wait hides its latency
#pragma unroll
    for (int r = 0; r < R; ++r) ubk[r] = tU[r * NT + tid];
    const bool first = k == K - 1, last = k == 0;
    // the next (earlier) iteration's pass bits and theta, for the a_t it will read
    const uint32_t bn = k > 0 ? tapeM[(size_t)(k - 1) * NT + tid] : 0u;
    const float opn = k > 0 ? 1.0f + A.coef[k - 1].th : 0.0f;
    float Ad[R];
    // reverse u-step: Au' = Au - div(pc a_t); the band's last row first (row below)
    auto ru_px = [&](int r) {
      const int lr = lr0 + r;
      const float at_top = (bits >> r) & 1u ? AP1[r] + opq * AQ1[r] : 0.0f;
      float at_bot;
      if (r == rb) at_bot = atB;
      else if (r + 1 < R) at_bot = (bits >> (r + 1)) & 1u ? AP1[r + 1] + opq * AQ1[r + 1] : 0.0f;
      else if (ty + 1 < TR) at_bot = sQ1[(ty + 1) * BW + j];
      else at_bot = sQ1h[j];
      const float at_left = (bits >> (8 + r)) & 1u ? AP2[r] + opq * AQ2[r] : 0.0f;
      const float at_right = sQ2[lr * L::QS + j + 1];
      const float dv = div_px(c.pc * at_top, c.pc * at_bot, c.pc * at_left, c.pc * at_right);
      const float aun = Au[r] - dv;
      float dub, df, dal;
      prox_partials_fg<FID>(ubk[r], sF[lr * BW + j], MASK && ((in_d >> r) & 1u), A.c1, A.c2, c, dub, df, dal);
      const float aub = dub * aun;
      Au[r] = aub;
      Ad[r] = c.sig * aub;
      sU[lr * L::US + j + 1] = Ad[r];
      if (df != 0.0f) Afr[r] += df * aun;
      if (col_ok && i0 + r < mr) {
        const float y = dal * aun - acc_c;
        const float tsum = acc_s + y;
        acc_c = (tsum - acc_s) - y;
        acc_s = tsum;
      }
    };
    if (CL > 1) cl_wait();
    ru_px(R - 1);
    if (push_down) st_remote(remote_uh, Ad[R - 1]);
    if (CL > 1) {
      if (push_down) cl_arrive<true>(); else cl_arrive<false>();
    }
#pragma unroll
    for (int r = 0; r + 1 < R; ++r) ru_px(r);
    __syncthreads();
    // reverse p-step; the band's first row first (row above)
    auto rp_px = [&](int r) {
      const int lr = lr0 + r;
      float ad_above;
      if (r > 0) ad_above = Ad[r - 1];
      else if (ty > 0) ad_above = sU[(lr - 1) * L::US + j + 1];
      else ad_above = sUh[j + 1];                      // 0 above the tile's first row
      const float ad_left = sU[lr * L::US + j];      // 0 left of the tile's first column
      adj_dof_reg(AP1[r], AQ1[r], AH1[r], (bits >> r) & 1u, ad_above - Ad[r], c, opq, first, last);
      adj_dof_reg(AP2[r], AQ2[r], AH2[r], (bits >> (8 + r)) & 1u, ad_left - Ad[r], c, opq, first, last);
      // a_t of the p2 dof for iteration k-1 (the left neighbour has read iteration k's)
      if (k > 0 && col_ok) sQ2[lr * L::QS + j] = ((bn >> (8 + r)) & 1u) ? AP2[r] + opn * AQ2[r] : 0.0f;
      if (r == rb && s_bot) {
        adj_dof_reg(APB, AQB, AHB, (bits >> 16) & 1u, Ad[r], c, opq, first, last);
        if (k > 0) atB = ((bn >> 16) & 1u) ? APB + opn * AQB : 0.0f;
      }
      if (right_thr) {
        float ap = sPR[lr], aq = sHR[lr], ah = sXR[lr];
        adj_dof_reg(ap, aq, ah, (bits >> (17 + r)) & 1u, Ad[r], c, opq, first, last);
        sPR[lr] = ap;
        sHR[lr] = aq;
        sXR[lr] = ah;
        if (k > 0) sQ2[lr * L::QS + mc] = ((bn >> (17 + r)) & 1u) ? ap + opn * aq : 0.0f;
      }
    };
    if (CL > 1) cl_wait();
    rp_px(0);
    if (k > 0) {  // row 0's a_t for iteration k-1 feeds the thread row / CTA above
      const float at10 = (bn & 1u) ? AP1[0] + opn * AQ1[0] : 0.0f;
      sQ1[ty * BW + j] = at10;
      if (push_up) st_remote(remote_q1h, at10);
    }
    if (CL > 1) {
      if (push_up) cl_arrive<true>(); else cl_arrive<false>();
    }
#pragma unroll
    for (int r = 1; r < R; ++r) rp_px(r);
    __syncthreads();  // every thread has read the Ad of its neighbours and published its a_t
  }
  if (CL > 1) cl_wait();

  // ---- store: Au, AP (folded), APhat on the subdomain's sides; Af += ; alpha partials
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const int i = i0 + r;
    if (!(col_ok && i < mr)) continue;
    const int gi = r0 + i;
    const size_t px = (size_t)gi * g.W + gj;
    Z.Au[px] = Au[r];
    if (Afr[r] != 0.0f) Z.Af[px] += Afr[r];
    const size_t e1 = (size_t)(gi + a) * g.W + gj, e2 = (size_t)gi * W2 + gj + b;
    if (i > 0 || s_top) Z.AP1[e1] = AP1[r];
    if (j > 0 || s_lft) Z.AP2[e2] = AP2[r];
    if (i == 0 && s_top) Z.APh1[e1] = AH1[r];
    if (j == 0 && s_lft) Z.APh2[e2] = AH2[r];
    if (i == mr - 1 && s_bot) {
      Z.AP1[e1 + g.W] = APB;
      Z.APh1[e1 + g.W] = AHB;
    }
    if (right_thr) {
      Z.AP2[e2 + 1] = sPR[lr0 + r];
      Z.APh2[e2 + 1] = sXR[lr0 + r];
    }
  }
  double acc = (double)acc_s - (double)acc_c;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  __shared__ double sw[NT / 32];
  if ((tid & 31) == 0) sw[tid >> 5] = acc;
  __syncthreads();
  if (tid == 0) {
    double t = 0.0;
    for (int w = 0; w < NT / 32; ++w) t += sw[w];
    Z.Aal[((size_t)a * g.NC + b) * CL + rank] += t;
  }
}

// ---------------------------------------------------------------------------
// The same reverse pass for subdomains of exactly 128 x 128 pixels, with the halo
// exchange of the persistent forward kernels (kernels_fused_mt.cu): a halo row is stored
// into the neighbour CTA with st.async and counted on an mbarrier there; only the
// warps that read a halo wait for it (bounded), and no cluster barrier runs inside the
// loops.  The reverse iteration has the forward's pattern, so the two barriers go on
// counting phases: the u halo (forward u, reverse Ad) travels down, the pbar1 halo
// (forward pbar1, reverse a_t of the first row) travels up.  No per-pixel validity test
// is needed: every thread owns 8 rows of one column.  Arithmetic and operation order
// are those of k_adj_fused (same bits).
template <int R, int TR>
struct AdjFullLayout {
  using F = FullLayout<R, TR>;
  static constexpr int XR = F::FLOATS;             // BAND: right-side adjoint of phat
  static constexpr int MB = (XR + TR * R + 1) & ~1;  // mbU, mbQ
  static constexpr size_t BYTES = sizeof(float) * MB + 16;
  static constexpr size_t tape_floats(int K) { return (size_t)K * (R + 1) * (128 * TR); }
};

template <int R, int TR, int CL, int MINB, int FID, bool MASK>
__global__ void __launch_bounds__(128 * TR, MINB) k_adj_full(const LocalArgs A, const AdjArgs Z) {
  using L = FullLayout<R, TR>;
  using AL = AdjFullLayout<R, TR>;
  constexpr int BW = L::BW, BAND = L::BAND, NT = BW * TR;
  static_assert(CL * BAND == 128 && CL > 1, "a cluster of CTAs covers the 128 rows of a tile");
  static_assert(R <= 8, "pass-bit word layout");
  extern __shared__ __align__(16) float smem[];
  float* sU = smem + L::U;
  float* sQ2 = smem + L::Q2;
  float* sQ1 = smem + L::Q1;
  float* sF = smem + L::F;
  float* sPR = smem + L::PR;
  float* sHR = smem + L::HR;
  float* sCo = smem + L::CO;
  float* sXR = smem + AL::XR;
  const uint32_t mbU = smem_addr(smem + AL::MB);
  const uint32_t mbQ = mbU + 8;

  const Grid g = A.g;
  const int K = A.K;
  const int rank = (int)blockIdx.x;
  const int b = blockIdx.y, a = blockIdx.z;
  const int r0 = a * 128, c0 = b * 128;
  const bool s_top = a > 0, s_bot = a + 1 < g.NR, s_lft = b > 0, s_rgt = b + 1 < g.NC;
  const int j = threadIdx.x, ty = threadIdx.y, tid = ty * BW + j;
  const int lr0 = ty * R;
  const int i0 = rank * BAND + lr0;
  const int W2 = g.W + g.NC;
  const int gj = c0 + j;
  const float tau = A.tau;
  const float lim_left = (j == 0 && !s_lft) ? 0.f : 1.f;
  const float lim_top = (i0 == 0 && !s_top) ? 0.f : 1.f;
  const bool last_row_here = rank == CL - 1 && ty == TR - 1;
  const bool push_down = ty == TR - 1 && rank + 1 < CL;  // last row -> u / Ad halo of rank + 1
  const bool push_up = ty == 0 && rank > 0;              // first row -> pbar1 / a_t halo of rank - 1
  const bool need_uh = push_up, need_qh = push_down;
  const bool right_lane = s_rgt && j < R;                // the right side of band row lr0 + j
  constexpr uint32_t kHaloBytes = 4 * BW;
  float* tapeU = Z.tape + ((size_t)(a * g.NC + b) * CL + rank) * AL::tape_floats(K);
  uint32_t* tapeM = reinterpret_cast<uint32_t*>(tapeU + (size_t)K * R * NT);
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
  bool timed_out = false;
  uint32_t phU = 0, phQ = 0;
  auto wait_u = [&]() {
    if (j == 0) mbar_arrive_expect_tx(mbU, kHaloBytes);
    if (!mbar_wait(mbU, phU & 1u)) timed_out = true;
    ++phU;
  };
  auto wait_q = [&]() {
    if (j == 0) mbar_arrive_expect_tx(mbQ, kHaloBytes);
    if (!mbar_wait(mbQ, phQ & 1u)) timed_out = true;
    ++phQ;
  };

  float u[R], p1[R], p2[R], h1[R], h2[R], q1[R];
  uint32_t in_d = 0;
  float pB = 0.f, hB = 0.f;
  for (int q = tid; q < 8 * min(K, L::kMaxSmemCoef); q += NT) sCo[q] = reinterpret_cast<const float*>(A.coef)[q];
  if (rank == 0) sU[1 + j] = 0.f;  // nothing above the tile's first row
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
  cluster_arrive<true>();  // barriers initialised everywhere before any halo is sent
  cluster_wait();
  if (push_up) st_cluster(remote_q1, q1[0]);  // the initial pbar1 halo, ordered by the barrier
  cluster_arrive<true>();
  cluster_wait();

  float* sUr = sU + (lr0 + 1) * L::US + j + 1;
  float* sQ2r = sQ2 + lr0 * L::QS + j;
  const float* sFr = sF + lr0 * BW + j;

  // ---- forward: K inner iterations, recording the tape
  for (int k = 0; k < K; ++k) {
    Coef c;
    if (k < L::kMaxSmemCoef) {
      const float4 ca = *reinterpret_cast<const float4*>(sCo + 8 * k);
      const float4 cb = *reinterpret_cast<const float4*>(sCo + 8 * k + 4);
      c = Coef{ca.x, ca.y, ca.z, ca.w, cb.x, cb.y, cb.z, cb.w};
    } else {
      c = A.coef[k];
    }
    float* tU = tapeU + (size_t)k * R * NT;
    if (need_qh && k > 0) wait_q();
#pragma unroll
    for (int rr = 0; rr < R; ++rr) {
      const int r = (rr + R - 1) % R;
      const float below = r + 1 < R ? q1[r + 1] : sQ1[(ty + 1) * BW + j];
      const float d = div_px(q1[r], below, sQ2r[r * L::QS], sQ2r[r * L::QS + 1]);
      const float ub = fmaf(c.sig, d, u[r]);
      tU[r * NT + tid] = ub;
      u[r] = prox_ubar<FID>(ub, sFr[r * BW], MASK && ((in_d >> r) & 1u), c);
      sUr[r * L::US] = u[r];
      if (rr == 0 && push_down) st_async_f32(remote_u, u[R - 1], remote_mbU);
    }
    __syncthreads();
    if (need_uh) wait_u();
    uint32_t bits = 0;
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const float above = r > 0 ? u[r - 1] : sUr[-L::US];
      bits |= p_step_bit(p1[r], q1[r], u[r] - above, h1[r], c, r == 0 ? lim_top : 1.f) << r;
      float q2;
      bits |= p_step_bit(p2[r], q2, u[r] - sUr[r * L::US - 1], h2[r], c, lim_left) << (8 + r);
      sQ2r[r * L::QS] = q2;
      if (r == 0) {
        sQ1[ty * BW + j] = q1[0];
        if (push_up) st_async_f32(remote_q1, q1[0], remote_mbQ);
      }
    }
    if (last_row_here && s_bot) {
      float qB;
      bits |= p_step_bit(pB, qB, -u[R - 1], hB, c, 1.f) << 16;
      sQ1[TR * BW + j] = qB;
    }
    if (right_lane) {
      const int lr = lr0 + j;
      float pr = sPR[lr], qr;
      bits |= p_step_bit(pr, qr, -sU[(lr + 1) * L::US + 128], sHR[lr], c, 1.f) << 17;
      sPR[lr] = pr;
      sQ2[lr * L::QS + 128] = qr;
    }
    tapeM[(size_t)k * NT + tid] = bits;
    __syncthreads();
  }
  if (need_qh) wait_q();  // the last forward pbar1 halo is not read
  // every forward halo has landed everywhere before the reverse sends its first ones
  // (otherwise two pushes into the same halo buffer could be in flight at once)
  cluster_arrive<true>();
  cluster_wait();

  // ---- reverse (registers: adjoints of u, p1, p2, pbar1, pbar2, phat1, phat2 and of
  // the bottom side; the right side's in sPR / sHR / sXR, handled by lane j for band
  // row lr0 + j; sU = Ad with row 0 the halo from above, sQ2 = a_t of the p2 dofs and
  // the right side, sQ1 = a_t of each thread row's first p1 row, row TR from below)
  float Au[R], AP1[R], AP2[R], AQ1[R], AQ2[R], AH1[R], AH2[R], Afr[R];
  float APB = 0.f, AQB = 0.f, AHB = 0.f;
  // the thread's share of dL/dalpha: compensated float32 sum (Kahan) over its pixels and
  // the K reverse iterations, then float64 across threads (a float64 operation per pixel
  // and iteration made this kernel wait on the slow float64 pipe)
  float acc_s = 0.f, acc_c = 0.f;
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const int gi = r0 + i0 + r;
    Au[r] = Z.Au[(size_t)gi * g.W + gj];
    AP1[r] = Z.AP1[(size_t)(gi + a) * g.W + gj];
    AP2[r] = Z.AP2[(size_t)gi * W2 + gj + b];
    AQ1[r] = AQ2[r] = AH1[r] = AH2[r] = Afr[r] = 0.f;
  }
  if (last_row_here && s_bot) APB = Z.AP1[(size_t)(r0 + 128 + a) * g.W + gj];
  if (right_lane) {
    sPR[lr0 + j] = Z.AP2[(size_t)(r0 + i0 + j) * W2 + c0 + 128 + b];
    sHR[lr0 + j] = 0.f;
    sXR[lr0 + j] = 0.f;
  }
  {
    const Coef c = A.coef[K - 1];
    const float opq = 1.0f + c.th;
    const uint32_t bits = tapeM[(size_t)(K - 1) * NT + tid];
#pragma unroll
    for (int r = 0; r < R; ++r) sQ2r[r * L::QS] = ((bits >> (8 + r)) & 1u) ? AP2[r] + opq * AQ2[r] : 0.0f;
    if (j < R) {
      const int lr = lr0 + j;
      sQ2[lr * L::QS + 128] = (right_lane && ((bits >> 17) & 1u)) ? sPR[lr] + opq * sHR[lr] : 0.0f;
    }
    const float at10 = (bits & 1u) ? AP1[0] + opq * AQ1[0] : 0.0f;
    sQ1[ty * BW + j] = at10;
    if (last_row_here) sQ1[TR * BW + j] = (s_bot && ((bits >> 16) & 1u)) ? APB + opq * AQB : 0.0f;
    __syncthreads();  // the forward's reads of sQ1 / sQ2 are over in this CTA
    if (push_up) st_async_f32(remote_q1, at10, remote_mbQ);
  }

  for (int k = K - 1; k >= 0; --k) {
    const Coef c = A.coef[k];
    const float opq = 1.0f + c.th;
    const uint32_t bits = tapeM[(size_t)k * NT + tid];
    const float* tU = tapeU + (size_t)k * R * NT;
    float ubk[R];
#pragma unroll
    for (int r = 0; r < R; ++r) ubk[r] = tU[r * NT + tid];
    const bool first = k == K - 1, last = k == 0;
    const uint32_t bn = k > 0 ? tapeM[(size_t)(k - 1) * NT + tid] : 0u;
    const float opn = k > 0 ? 1.0f + A.coef[k - 1].th : 0.0f;
    float Ad[R];
    if (need_qh) wait_q();  // a_t of the first row below, iteration k
#pragma unroll
    for (int rr = 0; rr < R; ++rr) {
      const int r = (rr + R - 1) % R;
      const float at_top = ((bits >> r) & 1u) ? AP1[r] + opq * AQ1[r] : 0.0f;
      const float at_bot = r + 1 < R ? (((bits >> (r + 1)) & 1u) ? AP1[r + 1] + opq * AQ1[r + 1] : 0.0f)
                                     : sQ1[(ty + 1) * BW + j];
      const float at_left = ((bits >> (8 + r)) & 1u) ? AP2[r] + opq * AQ2[r] : 0.0f;
      const float at_right = sQ2r[r * L::QS + 1];
      const float dv = div_px(c.pc * at_top, c.pc * at_bot, c.pc * at_left, c.pc * at_right);
      const float aun = Au[r] - dv;
      float dub, df, dal;
      prox_partials_fg<FID>(ubk[r], sFr[r * BW], MASK && ((in_d >> r) & 1u), A.c1, A.c2, c, dub, df, dal);
      const float aub = dub * aun;
      Au[r] = aub;
      Ad[r] = c.sig * aub;
      sUr[r * L::US] = Ad[r];
      if (df != 0.0f) Afr[r] += df * aun;
      {
        const float y = dal * aun - acc_c;
        const float tsum = acc_s + y;
        acc_c = (tsum - acc_s) - y;
        acc_s = tsum;
      }
      if (rr == 0 && push_down) st_async_f32(remote_u, Ad[R - 1], remote_mbU);
    }
    __syncthreads();
    if (need_uh) wait_u();  // Ad of the last row above, iteration k
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const float ad_above = r > 0 ? Ad[r - 1] : sUr[-L::US];
      const float ad_left = sUr[r * L::US - 1];
      adj_dof_reg(AP1[r], AQ1[r], AH1[r], (bits >> r) & 1u, ad_above - Ad[r], c, opq, first, last);
      adj_dof_reg(AP2[r], AQ2[r], AH2[r], (bits >> (8 + r)) & 1u, ad_left - Ad[r], c, opq, first, last);
      if (k > 0) sQ2r[r * L::QS] = ((bn >> (8 + r)) & 1u) ? AP2[r] + opn * AQ2[r] : 0.0f;
      if (r == 0 && k > 0) {
        const float at10 = (bn & 1u) ? AP1[0] + opn * AQ1[0] : 0.0f;
        sQ1[ty * BW + j] = at10;
        if (push_up) st_async_f32(remote_q1, at10, remote_mbQ);
      }
    }
    if (last_row_here && s_bot) {
      adj_dof_reg(APB, AQB, AHB, (bits >> 16) & 1u, Ad[R - 1], c, opq, first, last);
      if (k > 0) sQ1[TR * BW + j] = ((bn >> 16) & 1u) ? APB + opn * AQB : 0.0f;
    }
    if (right_lane) {
      const int lr = lr0 + j;
      float ap = sPR[lr], aq = sHR[lr], ah = sXR[lr];
      adj_dof_reg(ap, aq, ah, (bits >> 17) & 1u, sU[(lr + 1) * L::US + 128], c, opq, first, last);
      sPR[lr] = ap;
      sHR[lr] = aq;
      sXR[lr] = ah;
      if (k > 0) sQ2[lr * L::QS + 128] = ((bn >> 17) & 1u) ? ap + opn * aq : 0.0f;
    }
    __syncthreads();
  }
  if (timed_out) atomicOr(A.err, 1);
  cluster_arrive<true>();  // no CTA leaves while a neighbour may still write into it
  cluster_wait();

  // ---- store: Au, AP (folded), APhat on the subdomain's sides; Af += ; alpha partials
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const int gi = r0 + i0 + r;
    const size_t px = (size_t)gi * g.W + gj;
    Z.Au[px] = Au[r];
    if (Afr[r] != 0.0f) Z.Af[px] += Afr[r];
    const size_t e1 = (size_t)(gi + a) * g.W + gj, e2 = (size_t)gi * W2 + gj + b;
    if (i0 + r > 0 || s_top) Z.AP1[e1] = AP1[r];
    if (j > 0 || s_lft) Z.AP2[e2] = AP2[r];
    if (i0 + r == 0 && s_top) Z.APh1[e1] = AH1[r];
    if (j == 0 && s_lft) Z.APh2[e2] = AH2[r];
  }
  if (last_row_here && s_bot) {
    const size_t e = (size_t)(r0 + 128 + a) * g.W + gj;
    Z.AP1[e] = APB;
    Z.APh1[e] = AHB;
  }
  if (right_lane) {
    const size_t e = (size_t)(r0 + i0 + j) * W2 + c0 + 128 + b;
    Z.AP2[e] = sPR[lr0 + j];
    Z.APh2[e] = sXR[lr0 + j];
  }
  double acc = (double)acc_s - (double)acc_c;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  __shared__ double sw[NT / 32];
  if ((tid & 31) == 0) sw[tid >> 5] = acc;
  __syncthreads();
  if (tid == 0) {
    double t = 0.0;
    for (int w = 0; w < NT / 32; ++w) t += sw[w];
    Z.Aal[((size_t)a * g.NC + b) * CL + rank] += t;
  }
}

template <int R, int TR, int CL, int MINB, int FID, bool MASK>
cudaError_t launch_adj_full_one(const LocalArgs& a, const AdjArgs& z, cudaStream_t st) {
  using AL = AdjFullLayout<R, TR>;
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
  return cudaLaunchKernelEx(&cfg, k_adj_full<R, TR, CL, MINB, FID, MASK>, a, z);
}

template <int R, int TR, int CL, int MINB>
cudaError_t launch_adj_full(const LocalArgs& a, const AdjArgs& z, int fid, cudaStream_t st) {
  const bool m = a.mask != nullptr;
  switch (fid) {
    case FID_L2:
      return m ? launch_adj_full_one<R, TR, CL, MINB, FID_L2, true>(a, z, st)
               : launch_adj_full_one<R, TR, CL, MINB, FID_L2, false>(a, z, st);
    case FID_L1:
      return m ? launch_adj_full_one<R, TR, CL, MINB, FID_L1, true>(a, z, st)
               : launch_adj_full_one<R, TR, CL, MINB, FID_L1, false>(a, z, st);
    default: return launch_adj_full_one<R, TR, CL, MINB, FID_SEG, false>(a, z, st);
  }
}

template <int R, int TR, int CL, int MINB, int FID, bool MASK>
cudaError_t prepare_adj_full_one() {
  using AL = AdjFullLayout<R, TR>;
  return cudaFuncSetAttribute(k_adj_full<R, TR, CL, MINB, FID, MASK>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)AL::BYTES);
}

template <int R, int TR, int CL, int MINB>
cudaError_t prepare_adj_full() {
  cudaError_t e;
  if ((e = prepare_adj_full_one<R, TR, CL, MINB, FID_L2, false>()) != cudaSuccess) return e;
  if ((e = prepare_adj_full_one<R, TR, CL, MINB, FID_L2, true>()) != cudaSuccess) return e;
  if ((e = prepare_adj_full_one<R, TR, CL, MINB, FID_L1, false>()) != cudaSuccess) return e;
  if ((e = prepare_adj_full_one<R, TR, CL, MINB, FID_L1, true>()) != cudaSuccess) return e;
  return prepare_adj_full_one<R, TR, CL, MINB, FID_SEG, false>();
}

template <int BW, int R, int TR, int CL, int MINB, int FID, bool MASK>
cudaError_t launch_adj_one(const LocalArgs& a, const AdjArgs& z, cudaStream_t st) {
  using L = AdjLayout<BW, R, TR>;
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
  return cudaLaunchKernelEx(&cfg, k_adj_fused<BW, R, TR, CL, MINB, FID, MASK>, a, z);
}

template <int BW, int R, int TR, int CL, int MINB>
cudaError_t launch_adj_cfg(const LocalArgs& a, const AdjArgs& z, int fid, cudaStream_t st) {
  const bool m = a.mask != nullptr;
  switch (fid) {
    case FID_L2:
      return m ? launch_adj_one<BW, R, TR, CL, MINB, FID_L2, true>(a, z, st)
               : launch_adj_one<BW, R, TR, CL, MINB, FID_L2, false>(a, z, st);
    case FID_L1:
      return m ? launch_adj_one<BW, R, TR, CL, MINB, FID_L1, true>(a, z, st)
               : launch_adj_one<BW, R, TR, CL, MINB, FID_L1, false>(a, z, st);
    default: return launch_adj_one<BW, R, TR, CL, MINB, FID_SEG, false>(a, z, st);
  }
}

template <int BW, int R, int TR, int CL, int MINB, int FID, bool MASK>
cudaError_t prepare_adj_one() {
  using L = AdjLayout<BW, R, TR>;
  return cudaFuncSetAttribute(k_adj_fused<BW, R, TR, CL, MINB, FID, MASK>,
                              cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L::BYTES);
}

template <int BW, int R, int TR, int CL, int MINB>
cudaError_t prepare_adj_cfg() {
  cudaError_t e;
  if ((e = prepare_adj_one<BW, R, TR, CL, MINB, FID_L2, false>()) != cudaSuccess) return e;
  if ((e = prepare_adj_one<BW, R, TR, CL, MINB, FID_L2, true>()) != cudaSuccess) return e;
  if ((e = prepare_adj_one<BW, R, TR, CL, MINB, FID_L1, false>()) != cudaSuccess) return e;
  if ((e = prepare_adj_one<BW, R, TR, CL, MINB, FID_L1, true>()) != cudaSuccess) return e;
  return prepare_adj_one<BW, R, TR, CL, MINB, FID_SEG, false>();
}

// configuration for a tile shape: 0 = up to 32 x 32 (CL 1), 1 = up to 64 x 64 (CL 1),
// 2 = up to 128 x 128 (cluster of 8); -1 if the tile is larger
int adj_pick(int mr, int mc) {
  if (mc <= 32 && mr <= 32) return 0;
  if (mc <= 64 && mr <= 64) return 1;
  if (mc <= 128 && mr <= 128) return 2;
  return -1;
}

}  // namespace

long long adj_alpha_slots_fused(const Grid& g) { return (long long)g.NR * g.NC * 8; }

size_t adj_fused_tape_floats(const Grid& g, int K) {
  const int mr = (g.H + g.NR - 1) / g.NR, mc = (g.W + g.NC - 1) / g.NC;
  const size_t tiles = (size_t)g.NR * g.NC;
  switch (adj_pick(mr, mc)) {
    case 0: return tiles * AdjLayout<32, 8, 4>::tape_floats(K);
    case 1: return tiles * AdjLayout<64, 8, 8>::tape_floats(K);
    case 2: return tiles * 8 * AdjLayout<128, 8, 2>::tape_floats(K);
    default: return 0;
  }
}

cudaError_t adj_fused_prepare() {
  cudaError_t e;
  if ((e = prepare_adj_full<8, 2, 8, 2>()) != cudaSuccess) return e;
  if ((e = prepare_adj_cfg<32, 8, 4, 1, 1>()) != cudaSuccess) return e;
  if ((e = prepare_adj_cfg<64, 8, 8, 1, 1>()) != cudaSuccess) return e;
  return prepare_adj_cfg<128, 8, 2, 8, 2>();
}

cudaError_t launch_adj_fused(const LocalArgs& a, const AdjArgs& z, int fid, cudaStream_t st) {
  if (a.g.H == 128 * a.g.NR && a.g.W == 128 * a.g.NC)  // every subdomain exactly 128 x 128
    return launch_adj_full<8, 2, 8, 2>(a, z, fid, st);
  const int mr = (a.g.H + a.g.NR - 1) / a.g.NR, mc = (a.g.W + a.g.NC - 1) / a.g.NC;
  switch (adj_pick(mr, mc)) {
    case 0: return launch_adj_cfg<32, 8, 4, 1, 1>(a, z, fid, st);
    case 1: return launch_adj_cfg<64, 8, 8, 1, 1>(a, z, fid, st);
    case 2: return launch_adj_cfg<128, 8, 2, 8, 2>(a, z, fid, st);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace ddtv
