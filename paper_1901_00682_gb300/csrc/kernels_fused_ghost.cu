// Persistent fused local solver with one halo exchange per inner iteration.
//
// The persistent asynchronous kernel (kernels_fused.cu, fused_pa_body) exchanges two
// halo rows per inner iteration between the CTAs of a subdomain's cluster: the u row
// after the u-step (for the p-step of the CTA below) and the pbar1 row after the
// p-step (for the u-step of the CTA above), two dependent cross-SM hops per iteration.
// Here every CTA except the first also computes the u-step of the row just above its
// band (the last row of the CTA above; a "ghost" row): it needs that row's u, f and
// its pbar1 and pbar2 values, and the pbar1 of the CTA's own first row.  So the only
// exchange per inner iteration happens after the p-step: each CTA sends its last row's
// pbar1 and pbar2 (with the right side's) down, and its first row's pbar1 up; both are
// consumed in the next iteration's u-step, by the last computations of the warps that
// need them, so the hop overlaps the u-step of the other rows.  The ghost row's u is
// computed with the same operations on the same values as the CTA that owns the row
// (the same bits), so the iteration is unchanged.
//
// A CTA may run one inner iteration ahead of a neighbour (each depends on the other's
// previous iteration only), so the halo arrays and their mbarriers are double-buffered
// by the parity of the iteration that produced them; the consumer re-arms a buffer's
// mbarrier as soon as it has waited on it, and the next write into that buffer comes
// after data the consumer sent later, so the bytes always land in an armed phase.
// Waits are bounded: when one runs out, the kernel sets the error flag.
#include "fused_common.cuh"
#include "internal.cuh"

namespace ddtv {

namespace {

template <int R, int TR>
struct PgLayout {
  using F = FullLayout<R, TR>;
  static constexpr int NT = 128 * TR;
  static constexpr int ST = (F::FLOATS + 3) & ~3;  // staging [field][r][thread]: u, f, p1, p2
  static constexpr int SX = ST + 4 * R * NT;       // extras [x][thread]
  // extras: 0 lamh above, 1 P1 bottom side, 2 lamh below, 3..3+R-1 lamv left, 3+R P2 right
  // side, 4+R lamv right, 5+R initial pbar1 of the row below the band, ghost row: 6+R u,
  // 7+R f, 8+R pbar1 (top edge), 9+R pbar2 (left edge), 10+R pbar2 of its right side
  static constexpr int NX = 11 + R;
  static constexpr int GHS = 260;                  // one ghost buffer: pbar1[128], pbar2[129]
  static constexpr int GH = SX + NX * NT;          // [2][GHS] ghost halo
  static constexpr int QH = GH + 2 * GHS;          // [2][128] pbar1 of the row below the band
  static constexpr int MB = (QH + 2 * 128 + 1) & ~1;  // mbG[2], mbQ[2]
  static constexpr size_t BYTES = sizeof(float) * MB + 32;
};

template <int R, int TR, int CL, int FID, bool MASK>
__device__ __forceinline__ void fused_pg_body(const LocalArgs& A, const int first, const int stride) {
  using L = FullLayout<R, TR>;
  using P = PgLayout<R, TR>;
  constexpr int BW = L::BW, BAND = L::BAND, NT = P::NT, H2 = R / 2;
  static_assert(CL * BAND == 128 && CL > 1, "a cluster of CTAs covers the 128 rows of a tile");
  static_assert(R % 2 == 0, "rows are paired");
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
  float* sGh = smem + P::GH;
  float* sQh = smem + P::QH;
  const uint32_t mb0 = smem_addr(smem + P::MB);
  auto mbG = [&](int q) { return mb0 + 8u * q; };
  auto mbQ = [&](int q) { return mb0 + 16u + 8u * q; };

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
  const bool go = ty == 0 && rank > 0;                 // computes the ghost row above the band
  const bool need_qh = ty == TR - 1 && rank + 1 < CL;  // reads the pbar1 row below the band
  const bool push_up = go;                             // first row's pbar1 -> CTA above
  const bool push_down = need_qh;                      // last row's pbar1, pbar2 -> CTA below
  constexpr uint32_t kQBytes = 4 * BW, kGBytes = 4 * (2 * BW + 1);
  // remote addresses of buffer 0; buffer 1 is at a fixed offset (kept in registers)
  uint32_t rq = 0, rmq = 0, rg1 = 0, rg2 = 0, rmg = 0;
  if (push_up) {
    rq = map_rank(smem_addr(sQh + j), rank - 1);
    rmq = map_rank(mbQ(0), rank - 1);
  }
  if (push_down) {
    rg1 = map_rank(smem_addr(sGh + j), rank + 1);
    rg2 = map_rank(smem_addr(sGh + BW + j), rank + 1);
    rmg = map_rank(mbG(0), rank + 1);
  }
  constexpr uint32_t kQBuf = 4u * 128, kGBuf = 4u * P::GHS;  // byte offset of buffer 1
  if (tid == 0) {
    for (int q = 0; q < 4; ++q) mbar_init(mb0 + 8u * q, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  for (int q = tid; q < 8 * min(K, L::kMaxSmemCoef); q += NT) sCo[q] = reinterpret_cast<const float*>(A.coef)[q];
  if (ty == 0) sU[1 + j] = 0.f;  // the band's row above in sU stays 0 (the tile's top; ghosts use u_g)
  if (j == 0) sU[0] = 0.f;
  __syncthreads();
  if (j == 0) {  // arm both buffers' first phases of the barriers this CTA consumes
    if (go) {
      mbar_arrive_expect_tx(mbG(0), kGBytes);
      mbar_arrive_expect_tx(mbG(1), kGBytes);
    }
    if (need_qh) {
      mbar_arrive_expect_tx(mbQ(0), kQBytes);
      mbar_arrive_expect_tx(mbQ(1), kQBytes);
    }
  }
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
    if (go) {
      const int gg = r0 + i0 - 1;  // the ghost row (the CTA above's last row)
      cp_async4(stx + (6 + R) * NT + tid, A.u + (size_t)gg * g.W + gj);
      cp_async4(stx + (7 + R) * NT + tid, A.f + (size_t)gg * g.W + gj);
      cp_async4(stx + (8 + R) * NT + tid, A.P1 + (size_t)(gg + a) * g.W + gj);
      cp_async4(stx + (9 + R) * NT + tid, A.P2 + (size_t)gg * W2 + gj + b);
      if (j == 0 && b + 1 < g.NC) cp_async4(stx + (10 + R) * NT + tid, A.P2 + (size_t)gg * W2 + c0 + 128 + b);
    }
    cp_async_commit();
  };

  bool timed_out = false;
  // parity bits of the next phase of each buffer's barrier this CTA waits for (bit q)
  uint32_t phG = 0, phQ = 0;
  auto wait_q = [&](int q) {
    if (!mbar_wait(mbQ(q), (phQ >> q) & 1u)) timed_out = true;
    phQ ^= 1u << q;
    if (j == 0) mbar_arrive_expect_tx(mbQ(q), kQBytes);  // arm the buffer's next phase
  };
  auto wait_g = [&](int q) {
    if (!mbar_wait(mbG(q), (phG >> q) & 1u)) timed_out = true;
    phG ^= 1u << q;
    if (j == 0) mbar_arrive_expect_tx(mbG(q), kGBytes);
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
    float pB = 0.f, hB = 0.f, qB = 0.f;
    float u_g = 0.f, f_g = 0.f;
    bool in_d_g = false;

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
    if (last_row_here && s_bot) {
      pB = stx[1 * NT + tid];
      hB = phat_s(pB, stx[2 * NT + tid], tau);
    }
    qB = pB;
    if (need_qh) sQh[1 * 128 + j] = stx[(5 + R) * NT + tid];  // "iteration -1": the initial state
    if (go) {
      u_g = stx[(6 + R) * NT + tid];
      f_g = stx[(7 + R) * NT + tid];
      if (FID == FID_SEG) f_g = (f_g - A.c1) * (f_g - A.c1) - (f_g - A.c2) * (f_g - A.c2);
      in_d_g = MASK && A.mask[(size_t)(r0 + i0 - 1) * g.W + gj];
      sGh[1 * P::GHS + j] = stx[(8 + R) * NT + tid];
      sGh[1 * P::GHS + BW + j] = stx[(9 + R) * NT + tid];
      if (j == 0) sGh[1 * P::GHS + 2 * BW] = s_rgt ? stx[(10 + R) * NT + tid] : 0.f;
    }
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
      const int hb = (k + 1) & 1;  // buffer holding the halo of iteration k - 1 (k = 0: the initial state)
      const f32x2 SIG = pk2(c.sig, c.sig), UA = pk2(c.ua, c.ua), UB = pk2(c.ub, c.ub);
      const f32x2 PA = pk2(c.pa, c.pa), PC = pk2(c.pc, c.pc), PB = pk2(c.pb, c.pb), TH = pk2(c.th, c.th);
      // u-step on row pairs; the pair holding the band's last row (which may need the
      // halo from below) last
      auto u_pair = [&](int i, f32x2 below) {
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
      };
#pragma unroll
      for (int i = 0; i + 1 < H2; ++i) u_pair(i, Q1v[i + 1]);
      if (need_qh && k > 0) wait_q(hb);  // pbar1 row below, iteration k - 1
      {
        const float below_last = need_qh ? sQh[hb * 128 + j] : (last_row_here ? qB : sQ1[(ty + 1) * BW + j]);
        u_pair(H2 - 1, pk2(hi2(Q1v[0]), below_last));
      }
      if (go) {  // the ghost row: the same operations as its owner's u-step
        if (k > 0) wait_g(hb);
        const float* gq = sGh + hb * P::GHS;
        const float d = div_px(gq[j], lo2(Q1v[0]), gq[BW + j], gq[BW + j + 1]);
        u_g = u_update<FID>(u_g, d, f_g, in_d_g, c);
      }
      __syncthreads();
      // p-step on row pairs; the pair holding the band's first row first
      float q2_last = 0.f;
#pragma unroll
      for (int i = 0; i < H2; ++i) {
        const f32x2 above = i > 0 ? U[i - 1] : pk2(go ? u_g : sUr[-L::US], lo2(U[H2 - 1]));
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
          if (i == H2 - 1) q2_last = hi2(q2);
        }
        if (i == 0) {
          const float q10 = lo2(Q1v[0]);
          sQ1[ty * BW + j] = q10;
          if (push_up) st_async_f32(rq + (k & 1) * kQBuf, q10, rmq + 8u * (k & 1));
        }
      }
      if (push_down) {
        st_async_f32(rg1 + (k & 1) * kGBuf, hi2(Q1v[H2 - 1]), rmg + 8u * (k & 1));
        st_async_f32(rg2 + (k & 1) * kGBuf, q2_last, rmg + 8u * (k & 1));
      }
      if (last_row_here && s_bot) p_update(pB, qB, -hi2(U[H2 - 1]), hB, c);
      float qr_last = 0.f;
      if (right_lane) {
        const int lr = lr0 + j;
        float pr = sPR[lr], qr;
        p_update(pr, qr, -sU[(lr + 1) * L::US + 128], sHR[lr], c);
        sPR[lr] = pr;
        sQ2[lr * L::QS + 128] = qr;
        qr_last = qr;
      }
      // the right side of the band's last row (0 on the image boundary)
      if (push_down && j == R - 1) st_async_f32(rg2 + (k & 1) * kGBuf + 4u * (BW - j), qr_last, rmg + 8u * (k & 1));
      __syncthreads();
    }
    if (need_qh) wait_q((K - 1) & 1);  // drain the last halos (not read)
    if (go) wait_g((K - 1) & 1);
#pragma unroll
    for (int i = 0; i < H2; ++i) {
      u[i] = lo2(U[i]);
      u[i + H2] = hi2(U[i]);
      p1[i] = lo2(P1v[i]);
      p1[i + H2] = hi2(P1v[i]);
      p2[i] = lo2(P2v[i]);
      p2[i + H2] = hi2(P2v[i]);
    }

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

template <int R, int TR, int CL, int MINB, int FID, bool MASK>
__global__ void __launch_bounds__(128 * TR, MINB) k_fused_pg(const LocalArgs A) {
  fused_pg_body<R, TR, CL, FID, MASK>(A, blockIdx.y, gridDim.y);
}

template <int R, int TR, int CL, int MINB, int FID, bool MASK>
int& pg_clusters(int dev) {
  static int n[64] = {0};
  return n[dev & 63];
}

template <int R, int TR, int CL, int MINB, int FID, bool MASK>
cudaError_t prepare_pg_one() {
  using P = PgLayout<R, TR>;
  auto kern = k_fused_pg<R, TR, CL, MINB, FID, MASK>;
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
  pg_clusters<R, TR, CL, MINB, FID, MASK>(dev) = n;
  return cudaSuccess;
}

template <int R, int TR, int CL, int MINB, int FID, bool MASK>
cudaError_t launch_pg_one(const LocalArgs& a, cudaStream_t st) {
  using P = PgLayout<R, TR>;
  int dev = 0;
  cudaGetDevice(&dev);
  const int tiles = a.g.NR * a.g.NC;
  int nc = pg_clusters<R, TR, CL, MINB, FID, MASK>(dev);
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
  return cudaLaunchKernelEx(&cfg, k_fused_pg<R, TR, CL, MINB, FID, MASK>, a);
}

}  // namespace

cudaError_t fused_pg_prepare() {
  cudaError_t e;
  if ((e = prepare_pg_one<8, 2, 8, 2, FID_L2, false>()) != cudaSuccess) return e;
  if ((e = prepare_pg_one<8, 2, 8, 2, FID_L2, true>()) != cudaSuccess) return e;
  if ((e = prepare_pg_one<8, 2, 8, 2, FID_L1, false>()) != cudaSuccess) return e;
  if ((e = prepare_pg_one<8, 2, 8, 2, FID_L1, true>()) != cudaSuccess) return e;
  return prepare_pg_one<8, 2, 8, 2, FID_SEG, false>();
}

cudaError_t launch_fused_pg(const LocalArgs& a, int fid, cudaStream_t st) {
  const bool m = a.mask != nullptr;
  switch (fid) {
    case FID_L2: return m ? launch_pg_one<8, 2, 8, 2, FID_L2, true>(a, st) : launch_pg_one<8, 2, 8, 2, FID_L2, false>(a, st);
    case FID_L1: return m ? launch_pg_one<8, 2, 8, 2, FID_L1, true>(a, st) : launch_pg_one<8, 2, 8, 2, FID_L1, false>(a, st);
    default: return launch_pg_one<8, 2, 8, 2, FID_SEG, false>(a, st);
  }
}

}  // namespace ddtv
