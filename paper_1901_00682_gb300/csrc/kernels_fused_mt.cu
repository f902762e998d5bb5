// Persistent fused local solver on 2 x 4 micro-tiles (128 x 128 subdomains).
//
// A mapping that gives each thread one column of R rows keeps vertical neighbours in
// registers, but every pixel trades its u and pbar2 with both neighbouring columns
// through shared memory in each inner iteration, about 39 bytes of shared-memory
// traffic per pixel and iteration.
// Here a thread owns a micro-tile of two adjacent columns and four rows.  Inside it
// every neighbour is in registers, and the micro-tile exchanges only its edges, each
// with one vector access per iteration:
//   * the u of its right column (the thread to the right reads it for the p2 step of
//     its left column),
//   * the pbar2 of its left edge (the thread to the left reads it for the u-step of
//     its right column),
//   * the u of its last row (for the thread row below),
//   * the pbar1 of its first row (for the thread row above),
// 11 bytes per pixel and iteration.  The pixel's f (or g) is read from shared memory
// as packed pairs.
//
// Rows are packed in pairs (r, r + 2) for the `*.f32x2` arithmetic; every value is
// computed with the operations of the scalar iteration (pointwise.cuh) in the same
// order, so the result is bit-identical to the other mappings.
//
// A CTA is 64 x 4 threads (tx: column pair, ty: thread row) holding a band of 16 rows;
// a cluster of 8 CTAs covers a subdomain and loops over subdomains (persistent),
// prefetching the next one with cp.async (16-byte copies for u, f and p1, whose rows
// stay 16-byte aligned in the torn layout; 4-byte copies for p2).  Halo rows between
// the CTAs of a cluster travel with st.async and mbarrier complete_tx (one mbarrier
// per halo direction, phases counted by both sides); every wait is bounded and a wait that runs out
// sets the error flag.  The tile's right side (the p2 dofs of column 128) is updated
// by lanes 0..3 of each thread row, its bottom side by the last thread row of the last
// CTA.
#include "fused_common.cuh"
#include "internal.cuh"

namespace ddtv {

namespace {

struct MtLayout {
  static constexpr int CL = 8, TR = 4, R = 4, NX = 64, NT = NX * TR, BAND = TR * R, BW = 128;
  static constexpr int P2S = 132;                    // staging row stride of p2 (129 values)
  static constexpr int SLOT = 4 * (NX + 1);          // one thread row of UR / QL
  // (TR + 1) x 128: row 0 = u of the row above the band (halo; zero in the first CTA),
  // row ty + 1 = u of the last row of thread row ty
  static constexpr int UB = 0;
  // (TR + 1) x 128: row ty = pbar1 of the first row of thread row ty, row TR = pbar1 of
  // the row below the band (halo, or the tile's bottom side)
  static constexpr int Q1 = UB + (TR + 1) * BW;
  // TR x (NX + 1) x 4: slot 0 = zero (left of the tile), slot tx + 1 = u of thread tx's
  // right column, rows in pair order (0, 2, 1, 3)
  static constexpr int UR = Q1 + (TR + 1) * BW;
  // TR x (NX + 1) x 4: slot tx = pbar2 of thread tx's left edge, slot NX = the tile's
  // right side; rows in pair order
  static constexpr int QL = UR + TR * SLOT;
  static constexpr int F = QL + TR * SLOT;           // TR x 2 x NX x 4: f (or g) of column 2tx + c, pair order
  static constexpr int PR = F + TR * 2 * NX * 4;     // BAND right-side p
  static constexpr int HR = PR + BAND;               // BAND right-side phat
  static constexpr int CO = HR + BAND;               // kMaxSmemCoef x 8 coefficients
  static constexpr int kMaxSmemCoef = 64;
  static constexpr int SU = CO + 16 * kMaxSmemCoef;  // staging of the next subdomain: u, f, p1 (BAND x 128 each)
  static constexpr int SP2 = SU + 3 * BAND * BW;     // p2 (BAND x P2S; column 128 = right side)
  static constexpr int XLT = SP2 + BAND * P2S;       // lamh above the tile (128)
  static constexpr int XPB = XLT + BW;               // p1 of the tile's bottom side (128)
  static constexpr int XLB = XPB + BW;               // lamh below the tile (128)
  static constexpr int XQH = XLB + BW;               // initial pbar1 of the row below the band (128)
  static constexpr int XLL = XQH + BW;               // lamv left of the band rows (BAND)
  static constexpr int XLR = XLL + BAND;             // lamv right of the band rows (BAND)
  static constexpr int MB = XLR + BAND;              // two mbarriers
  static constexpr size_t BYTES = sizeof(float) * MB + 16;
  static_assert(UR % 4 == 0 && QL % 4 == 0 && F % 4 == 0 && CO % 4 == 0 && SU % 4 == 0 && MB % 2 == 0,
                "vector accesses need 16-byte (mbarriers 8-byte) alignment");
  static_assert(CL * BAND == 128, "a cluster of CTAs covers the 128 rows of a tile");
};

// pair order of a micro-tile column: row r sits in pair r & 1, lane r >> 1
__device__ __forceinline__ float lane_of(f32x2 v, int h) { return h ? hi2(v) : lo2(v); }

template <int FID, bool MASK>
__device__ __forceinline__ void fused_mt_body(const LocalArgs& A, const int first, const int stride) {
  using L = MtLayout;
  constexpr int NX = L::NX, TR = L::TR, CL = L::CL, BAND = L::BAND, NT = L::NT, BW = L::BW;
  extern __shared__ __align__(16) float smem[];
  float* sUB = smem + L::UB;
  float* sQ1 = smem + L::Q1;
  float* sUR = smem + L::UR;
  float* sQL = smem + L::QL;
  float* sF = smem + L::F;
  float* sPR = smem + L::PR;
  float* sHR = smem + L::HR;
  float* sCo = smem + L::CO;
  const uint32_t mbU = smem_addr(smem + L::MB);
  const uint32_t mbQ = mbU + 8;

  const Grid g = A.g;
  const int T = g.NR * g.NC;
  const int rank = (int)blockIdx.x;
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int tid = ty * NX + tx;
  const int j0 = 2 * tx;             // the thread's first column in the tile
  const int lr0 = 4 * ty;            // its first row in the band
  const int i0 = rank * BAND + lr0;  // ... in the tile
  const int W2 = g.W + g.NC;
  const float tau = A.tau;
  const int K = A.K;
  const bool last_row_here = rank == CL - 1 && ty == TR - 1;
  const bool push_down = ty == TR - 1 && rank + 1 < CL;  // sends u of the band's last row
  const bool push_up = ty == 0 && rank > 0;              // sends pbar1 of the band's first row
  const bool need_uh = push_up;                          // p-step of thread row 0 reads the u row above
  const bool need_qh = push_down;                        // u-step of the last thread row reads pbar1 below
  constexpr uint32_t kHaloBytes = 4 * BW;
  float* const myUR = sUR + ty * L::SLOT + 4 * (tx + 1);
  float* const myQL = sQL + ty * L::SLOT + 4 * tx;
  uint32_t remote_u = 0, remote_q1 = 0, remote_mbU = 0, remote_mbQ = 0;
  if (push_down) {
    remote_u = map_rank(smem_addr(sUB + j0), rank + 1);
    remote_mbU = map_rank(mbU, rank + 1);
  }
  if (push_up) {
    remote_q1 = map_rank(smem_addr(sQ1 + TR * BW + j0), rank - 1);
    remote_mbQ = map_rank(mbQ, rank - 1);
  }
  if (tid == 0) {
    mbar_init(mbU, 1);
    mbar_init(mbQ, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  for (int q = tid; q < 8 * min(K, L::kMaxSmemCoef); q += NT) sCo[q] = reinterpret_cast<const float*>(A.coef)[q];
  if (rank == 0 && ty == 0) {  // u = 0 above every tile's first row
    sUB[j0] = 0.f;
    sUB[j0 + 1] = 0.f;
  }
  if (tx < 4) sUR[ty * L::SLOT + tx] = 0.f;  // u = 0 left of the tile's first column
  __syncthreads();
  if (need_uh && tx == 0) mbar_arrive_expect_tx(mbU, kHaloBytes);
  if (need_qh && tx == 0) mbar_arrive_expect_tx(mbQ, kHaloBytes);
  cluster_arrive<true>();  // barriers initialised and armed everywhere before any halo is sent
  cluster_wait();

  auto prefetch = [&](int t) {
    const int a = t / g.NC, b = t - a * g.NC;
    const int c0 = b * 128;
    const int gb = a * 128 + rank * BAND;  // image row of the band's first row
#pragma unroll
    for (int m = 0; m < 6; ++m) {  // u, f, p1: 3 x BAND rows x 32 chunks of 16 bytes
      const int fld = m >> 1;
      const int q = tid + NT * (m & 1);
      const int row = q >> 5, ch = q & 31;
      const float* base = fld == 0 ? A.u : (fld == 1 ? A.f : A.P1);
      const int grow = gb + row + (fld == 2 ? a : 0);
      cp_async16(smem + L::SU + fld * BAND * BW + row * BW + 4 * ch, base + (size_t)grow * g.W + c0 + 4 * ch);
    }
    {  // p2: two rows per warp, 129 values each
      const int w = tid >> 5, lane = tid & 31;
#pragma unroll
      for (int rr = 0; rr < 2; ++rr) {
        const int row = 2 * w + rr;
        const float* src = A.P2 + (size_t)(gb + row) * W2 + c0 + b;
#pragma unroll
        for (int s = 0; s < 5; ++s) {
          const int col = lane + 32 * s;
          if (col <= 128) cp_async4(smem + L::SP2 + row * L::P2S + col, src + col);
        }
      }
    }
    if (i0 == 0 && (a > 0 || g.cut_top)) {
      cp_async4(smem + L::XLT + j0, A.lamh + (ptrdiff_t)(a - 1) * g.W + c0 + j0);
      cp_async4(smem + L::XLT + j0 + 1, A.lamh + (ptrdiff_t)(a - 1) * g.W + c0 + j0 + 1);
    }
    if (last_row_here && (a + 1 < g.NR || g.cut_bot)) {
#pragma unroll
      for (int c = 0; c < 2; ++c) {
        cp_async4(smem + L::XPB + j0 + c, A.P1 + (size_t)(a * 128 + 128 + a) * g.W + c0 + j0 + c);
        cp_async4(smem + L::XLB + j0 + c, A.lamh + (size_t)a * g.W + c0 + j0 + c);
      }
    }
    if (tx == 0 && b > 0) {
#pragma unroll
      for (int r = 0; r < 4; ++r) cp_async4(smem + L::XLL + lr0 + r, A.lamv + (size_t)(b - 1) * g.H + gb + lr0 + r);
    }
    if (tx < 4 && b + 1 < g.NC) cp_async4(smem + L::XLR + lr0 + tx, A.lamv + (size_t)b * g.H + gb + lr0 + tx);
    if (need_qh) {
#pragma unroll
      for (int c = 0; c < 2; ++c) cp_async4(smem + L::XQH + j0 + c, A.P1 + (size_t)(gb + BAND + a) * g.W + c0 + j0 + c);
    }
    cp_async_commit();
  };

  bool timed_out = false;
  uint32_t phU = 0, phQ = 0;  // index of the next phase of mbU / mbQ this CTA waits for
  auto wait_u = [&]() {
    if (!mbar_wait(mbU, phU & 1)) timed_out = true;
    ++phU;
    if (tx == 0) mbar_arrive_expect_tx(mbU, kHaloBytes);  // arm the next phase
  };
  auto wait_q = [&]() {
    if (!mbar_wait(mbQ, phQ & 1)) timed_out = true;
    ++phQ;
    if (tx == 0) mbar_arrive_expect_tx(mbQ, kHaloBytes);
  };

  if (first < T) prefetch(first);

  for (int t = first; t < T; t += stride) {
    const int a = t / g.NC, b = t - a * g.NC;
    const int c0 = b * 128;
    const int gb = a * 128 + rank * BAND;
    const bool s_top = a > 0 || g.cut_top, s_bot = a + 1 < g.NR || g.cut_bot, s_lft = b > 0, s_rgt = b + 1 < g.NC;
    const float lim_left = (tx == 0 && !s_lft) ? 0.f : 1.f;
    const float lim_top = (i0 == 0 && !s_top) ? 0.f : 1.f;
    const bool right_lane = s_rgt && tx < 4;
    // pairs [column c][e]: rows (e, e + 2) of column j0 + c
    f32x2 U[2][2], P1[2][2], P2[2][2], H1[2][2], H2[2][2], Q1[2][2], Q2[2][2];
    uint32_t in_d = 0;  // bit 4c + r: pixel (row r, column j0 + c) lies in the inpainting domain
    float pB[2] = {0.f, 0.f}, hB[2] = {0.f, 0.f};

    cp_async_wait_all();
    __syncthreads();  // staging landed; the previous subdomain's shared arrays are free
    {
      float u[4][2], fv[4][2], p1[4][2], p2[4][2];
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        const float2 uu = *reinterpret_cast<const float2*>(smem + L::SU + (lr0 + r) * BW + j0);
        const float2 ff = *reinterpret_cast<const float2*>(smem + L::SU + BAND * BW + (lr0 + r) * BW + j0);
        const float2 q1 = *reinterpret_cast<const float2*>(smem + L::SU + 2 * BAND * BW + (lr0 + r) * BW + j0);
        const float2 q2 = *reinterpret_cast<const float2*>(smem + L::SP2 + (lr0 + r) * L::P2S + j0);
        u[r][0] = uu.x;
        u[r][1] = uu.y;
        fv[r][0] = ff.x;
        fv[r][1] = ff.y;
        p1[r][0] = q1.x;
        p1[r][1] = q1.y;
        p2[r][0] = q2.x;
        p2[r][1] = q2.y;
#pragma unroll
        for (int c = 0; c < 2; ++c) {
          if (FID == FID_SEG) fv[r][c] = (fv[r][c] - A.c1) * (fv[r][c] - A.c1) - (fv[r][c] - A.c2) * (fv[r][c] - A.c2);
          if (MASK && A.mask[(size_t)(gb + lr0 + r) * g.W + c0 + j0 + c]) in_d |= 1u << (4 * c + r);
        }
      }
      float h1[4][2], h2[4][2];
#pragma unroll
      for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int c = 0; c < 2; ++c) {
          h1[r][c] = p1[r][c];
          h2[r][c] = p2[r][c];
        }
      if (i0 == 0 && s_top) {
#pragma unroll
        for (int c = 0; c < 2; ++c) h1[0][c] = phat_t(p1[0][c], smem[L::XLT + j0 + c], tau);
      }
      if (tx == 0 && s_lft) {
#pragma unroll
        for (int r = 0; r < 4; ++r) h2[r][0] = phat_t(p2[r][0], smem[L::XLL + lr0 + r], tau);
      }
#pragma unroll
      for (int c = 0; c < 2; ++c)
#pragma unroll
        for (int e = 0; e < 2; ++e) {
          U[c][e] = pk2(u[e][c], u[e + 2][c]);
          P1[c][e] = pk2(p1[e][c], p1[e + 2][c]);
          P2[c][e] = pk2(p2[e][c], p2[e + 2][c]);
          H1[c][e] = pk2(h1[e][c], h1[e + 2][c]);
          H2[c][e] = pk2(h2[e][c], h2[e + 2][c]);
          Q1[c][e] = P1[c][e];
          Q2[c][e] = P2[c][e];
        }
#pragma unroll
      for (int c = 0; c < 2; ++c)
        *reinterpret_cast<ulonglong2*>(sF + ((ty * 2 + c) * NX + tx) * 4) =
            make_ulonglong2(pk2(fv[0][c], fv[2][c]), pk2(fv[1][c], fv[3][c]));
      *reinterpret_cast<ulonglong2*>(myQL) = make_ulonglong2(P2[0][0], P2[0][1]);
      *reinterpret_cast<float2*>(sQ1 + ty * BW + j0) = make_float2(p1[0][0], p1[0][1]);
      if (last_row_here) {
        if (s_bot) {
#pragma unroll
          for (int c = 0; c < 2; ++c) {
            pB[c] = smem[L::XPB + j0 + c];
            hB[c] = phat_s(pB[c], smem[L::XLB + j0 + c], tau);
          }
        }
        *reinterpret_cast<float2*>(sQ1 + TR * BW + j0) = make_float2(pB[0], pB[1]);
      }
      if (need_qh)
        *reinterpret_cast<float2*>(sQ1 + TR * BW + j0) = *reinterpret_cast<const float2*>(smem + L::XQH + j0);
      if (tx < 4) {
        const int lr = lr0 + tx;
        float pr = 0.f, hr = 0.f;
        if (s_rgt) {
          pr = smem[L::SP2 + lr * L::P2S + 128];
          hr = phat_s(pr, smem[L::XLR + lr], tau);
        }
        sPR[lr] = pr;
        sHR[lr] = hr;
        sQL[ty * L::SLOT + 4 * NX + (tx & 1) * 2 + (tx >> 1)] = pr;
      }
    }
    __syncthreads();  // staging consumed by every thread
    if (t + stride < T) prefetch(t + stride);

    for (int k = 0; k < K; ++k) {
      Coef co;
      if (k < L::kMaxSmemCoef) {
        const float4 ca = *reinterpret_cast<const float4*>(sCo + 8 * k);
        const float4 cb = *reinterpret_cast<const float4*>(sCo + 8 * k + 4);
        co = Coef{ca.x, ca.y, ca.z, ca.w, cb.x, cb.y, cb.z, cb.w};
      } else {
        co = A.coef[k];
      }
      const f32x2 SIG = pk2(co.sig, co.sig), UA = pk2(co.ua, co.ua), UB = pk2(co.ub, co.ub);
      const f32x2 PA = pk2(co.pa, co.pa), PC = pk2(co.pc, co.pc), PB = pk2(co.pb, co.pb), TH = pk2(co.th, co.th);
      if (need_qh && k > 0) wait_q();  // pbar1 halo of iteration k-1
      // ---- u-step: pair e = 1 (holding the thread's last row) first
      {
        const ulonglong2 qr = *reinterpret_cast<const ulonglong2*>(myQL + 4);  // left edge of the thread to the right
        const float2 qb = *reinterpret_cast<const float2*>(sQ1 + (ty + 1) * BW + j0);  // pbar1 of the row below
        const ulonglong2 fc0 = *reinterpret_cast<const ulonglong2*>(sF + ((ty * 2 + 0) * NX + tx) * 4);
        const ulonglong2 fc1 = *reinterpret_cast<const ulonglong2*>(sF + ((ty * 2 + 1) * NX + tx) * 4);
#pragma unroll
        for (int ee = 0; ee < 2; ++ee) {
          const int e = 1 - ee;
#pragma unroll
          for (int c = 0; c < 2; ++c) {
            const f32x2 below = e == 0 ? Q1[c][1] : pk2(hi2(Q1[c][0]), c == 0 ? qb.x : qb.y);
            const f32x2 right = c == 0 ? Q2[1][e] : (e == 0 ? qr.x : qr.y);
            const f32x2 d = sub2(add2(sub2(below, Q1[c][e]), right), Q2[c][e]);  // div_px
            const f32x2 fg = c == 0 ? (e == 0 ? fc0.x : fc0.y) : (e == 0 ? fc1.x : fc1.y);
            const f32x2 ub = fma2(SIG, d, U[c][e]);
            const bool dl = MASK && ((in_d >> (4 * c + e)) & 1u), dh = MASK && ((in_d >> (4 * c + e + 2)) & 1u);
            f32x2 un;
            if (FID == FID_L2) {
              un = fma2(UB, fg, mul2(UA, ub));
              if (MASK) un = pk2(dl ? lo2(ub) : lo2(un), dh ? hi2(ub) : hi2(un));
            } else {
              un = pk2(prox_ubar<FID>(lo2(ub), lo2(fg), dl, co), prox_ubar<FID>(hi2(ub), hi2(fg), dh, co));
            }
            U[c][e] = un;
          }
          if (e == 1 && push_down) st_async_v2(remote_u, hi2(U[0][1]), hi2(U[1][1]), remote_mbU);
        }
        *reinterpret_cast<ulonglong2*>(myUR) = make_ulonglong2(U[1][0], U[1][1]);
        if (ty < TR - 1) *reinterpret_cast<float2*>(sUB + (ty + 1) * BW + j0) = make_float2(hi2(U[0][1]), hi2(U[1][1]));
      }
      __syncthreads();
      if (need_uh) wait_u();  // u halo of iteration k
      // ---- p-step: pair e = 0 (holding the thread's first row) first
      {
        const float2 ua = *reinterpret_cast<const float2*>(sUB + ty * BW + j0);  // u of the row above
        const ulonglong2 ul = *reinterpret_cast<const ulonglong2*>(myUR - 4);    // right column of the thread to the left
#pragma unroll
        for (int e = 0; e < 2; ++e) {
#pragma unroll
          for (int c = 0; c < 2; ++c) {
            const f32x2 above = e == 1 ? U[c][0] : pk2(c == 0 ? ua.x : ua.y, lo2(U[c][1]));
            const f32x2 leftu = c == 1 ? U[0][e] : (e == 0 ? ul.x : ul.y);
            {
              const f32x2 tt = fma2(PC, sub2(U[c][e], above), fma2(PA, P1[c][e], mul2(PB, H1[c][e])));  // p_target
              const float l0 = e == 0 ? lim_top : 1.f;
              const f32x2 pn = pk2(clamp_abs(lo2(tt), l0), clamp_abs(hi2(tt), 1.f));
              Q1[c][e] = fma2(TH, sub2(pn, P1[c][e]), pn);
              P1[c][e] = pn;
            }
            {
              const f32x2 tt = fma2(PC, sub2(U[c][e], leftu), fma2(PA, P2[c][e], mul2(PB, H2[c][e])));
              const float l = c == 0 ? lim_left : 1.f;
              const f32x2 pn = pk2(clamp_abs(lo2(tt), l), clamp_abs(hi2(tt), l));
              Q2[c][e] = fma2(TH, sub2(pn, P2[c][e]), pn);
              P2[c][e] = pn;
            }
          }
          if (e == 0) {
            const float qa = lo2(Q1[0][0]), qc = lo2(Q1[1][0]);
            if (ty > 0) *reinterpret_cast<float2*>(sQ1 + ty * BW + j0) = make_float2(qa, qc);
            if (push_up) st_async_v2(remote_q1, qa, qc, remote_mbQ);
          }
        }
        *reinterpret_cast<ulonglong2*>(myQL) = make_ulonglong2(Q2[0][0], Q2[0][1]);
      }
      if (last_row_here && s_bot) {
#pragma unroll
        for (int c = 0; c < 2; ++c) {
          float qB;
          p_update(pB[c], qB, -hi2(U[c][1]), hB[c], co);
          sQ1[TR * BW + j0 + c] = qB;
        }
      }
      if (right_lane) {
        const int lr = lr0 + tx;
        const int pos = (tx & 1) * 2 + (tx >> 1);
        float pr = sPR[lr], qr;
        p_update(pr, qr, -sUR[ty * L::SLOT + 4 * NX + pos], sHR[lr], co);
        sPR[lr] = pr;
        sQL[ty * L::SLOT + 4 * NX + pos] = qr;
      }
      __syncthreads();
    }
    if (need_qh) wait_q();  // drain the last pbar1 halo (not read)

#pragma unroll
    for (int r = 0; r < 4; ++r) {
      const int e = r & 1, h = r >> 1;
      const int gi = gb + lr0 + r;
      *reinterpret_cast<float2*>(A.u + (size_t)gi * g.W + c0 + j0) = make_float2(lane_of(U[0][e], h), lane_of(U[1][e], h));
      *reinterpret_cast<float2*>(A.P1 + (size_t)(gi + a) * g.W + c0 + j0) =
          make_float2(lane_of(P1[0][e], h), lane_of(P1[1][e], h));
      float* p2row = A.P2 + (size_t)gi * W2 + c0 + b + j0;
      p2row[0] = lane_of(P2[0][e], h);
      p2row[1] = lane_of(P2[1][e], h);
    }
    if (i0 == 0 && s_top) {
      A.out.ST[(ptrdiff_t)(a - 1) * g.W + c0 + j0] = lo2(P1[0][0]);
      A.out.ST[(ptrdiff_t)(a - 1) * g.W + c0 + j0 + 1] = lo2(P1[1][0]);
    }
    if (tx == 0 && s_lft) {
#pragma unroll
      for (int r = 0; r < 4; ++r) A.out.SL[(size_t)(b - 1) * g.H + gb + lr0 + r] = lane_of(P2[0][r & 1], r >> 1);
    }
    if (last_row_here && s_bot) {
#pragma unroll
      for (int c = 0; c < 2; ++c) {
        A.P1[(size_t)(a * 128 + 128 + a) * g.W + c0 + j0 + c] = pB[c];
        A.out.SB[(size_t)a * g.W + c0 + j0 + c] = pB[c];
      }
    }
    if (right_lane) {
      const int gi = gb + lr0 + tx;
      const float pr = sPR[lr0 + tx];
      A.P2[(size_t)gi * W2 + c0 + 128 + b] = pr;
      A.out.SR[(size_t)b * g.H + gi] = pr;
    }
  }
  cp_async_wait_all();
  cluster_arrive<true>();  // no CTA leaves while a neighbour may still write into it
  cluster_wait();
  if (timed_out) atomicOr(A.err, 1);
}

// The same body over a source of subdomains (fused_common.cuh): BatchTiles runs the
// work list of a batch, each subdomain with its image's geometry, parameters, strips
// and fidelity, and the image's coefficients reloaded into shared memory when the
// image changes.  (The single-image kernel keeps its own copy above: compiled through
// this generic body it measured 5 % slower.)
template <bool MASK, class Src>
__device__ __forceinline__ void fused_mt_run(const Src& S, const int first, const int stride) {
  using L = MtLayout;
  constexpr int NX = L::NX, TR = L::TR, CL = L::CL, BAND = L::BAND, NT = L::NT, BW = L::BW;
  extern __shared__ __align__(16) float smem[];
  float* sUB = smem + L::UB;
  float* sQ1 = smem + L::Q1;
  float* sUR = smem + L::UR;
  float* sQL = smem + L::QL;
  float* sF = smem + L::F;
  float* sPR = smem + L::PR;
  float* sHR = smem + L::HR;
  float* sCo = smem + L::CO;
  const uint32_t mbU = smem_addr(smem + L::MB);
  const uint32_t mbQ = mbU + 8;

  const int T = S.count();
  const int rank = (int)blockIdx.x;
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int tid = ty * NX + tx;
  const int j0 = 2 * tx;             // the thread's first column in the tile
  const int lr0 = 4 * ty;            // its first row in the band
  const int i0 = rank * BAND + lr0;  // ... in the tile
  const int K = S.inner();
  const bool last_row_here = rank == CL - 1 && ty == TR - 1;
  const bool push_down = ty == TR - 1 && rank + 1 < CL;  // sends u of the band's last row
  const bool push_up = ty == 0 && rank > 0;              // sends pbar1 of the band's first row
  const bool need_uh = push_up;                          // p-step of thread row 0 reads the u row above
  const bool need_qh = push_down;                        // u-step of the last thread row reads pbar1 below
  constexpr uint32_t kHaloBytes = 4 * BW;
  float* const myUR = sUR + ty * L::SLOT + 4 * (tx + 1);
  float* const myQL = sQL + ty * L::SLOT + 4 * tx;
  uint32_t remote_u = 0, remote_q1 = 0, remote_mbU = 0, remote_mbQ = 0;
  if (push_down) {
    remote_u = map_rank(smem_addr(sUB + j0), rank + 1);
    remote_mbU = map_rank(mbU, rank + 1);
  }
  if (push_up) {
    remote_q1 = map_rank(smem_addr(sQ1 + TR * BW + j0), rank - 1);
    remote_mbQ = map_rank(mbQ, rank - 1);
  }
  if (tid == 0) {
    mbar_init(mbU, 1);
    mbar_init(mbQ, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  int cur_img = -1;  // image whose coefficients are in sCo
  if (rank == 0 && ty == 0) {  // u = 0 above every tile's first row
    sUB[j0] = 0.f;
    sUB[j0 + 1] = 0.f;
  }
  if (tx < 4) sUR[ty * L::SLOT + tx] = 0.f;  // u = 0 left of the tile's first column
  __syncthreads();
  if (need_uh && tx == 0) mbar_arrive_expect_tx(mbU, kHaloBytes);
  if (need_qh && tx == 0) mbar_arrive_expect_tx(mbQ, kHaloBytes);
  cluster_arrive<true>();  // barriers initialised and armed everywhere before any halo is sent
  cluster_wait();

  auto prefetch = [&](int t) {
    const LocalArgs& A = S.args(t);
    const Grid g = A.g;
    const int W2 = g.W + g.NC;
    const int lt = S.local(t);
    const int a = lt / g.NC, b = lt - a * g.NC;
    const int c0 = b * 128;
    const int gb = a * 128 + rank * BAND;  // image row of the band's first row
#pragma unroll
    for (int m = 0; m < 6; ++m) {  // u, f, p1: 3 x BAND rows x 32 chunks of 16 bytes
      const int fld = m >> 1;
      const int q = tid + NT * (m & 1);
      const int row = q >> 5, ch = q & 31;
      const float* base = fld == 0 ? A.u : (fld == 1 ? A.f : A.P1);
      const int grow = gb + row + (fld == 2 ? a : 0);
      cp_async16(smem + L::SU + fld * BAND * BW + row * BW + 4 * ch, base + (size_t)grow * g.W + c0 + 4 * ch);
    }
    {  // p2: two rows per warp, 129 values each
      const int w = tid >> 5, lane = tid & 31;
#pragma unroll
      for (int rr = 0; rr < 2; ++rr) {
        const int row = 2 * w + rr;
        const float* src = A.P2 + (size_t)(gb + row) * W2 + c0 + b;
#pragma unroll
        for (int s = 0; s < 5; ++s) {
          const int col = lane + 32 * s;
          if (col <= 128) cp_async4(smem + L::SP2 + row * L::P2S + col, src + col);
        }
      }
    }
    if (i0 == 0 && (a > 0 || g.cut_top)) {
      cp_async4(smem + L::XLT + j0, A.lamh + (ptrdiff_t)(a - 1) * g.W + c0 + j0);
      cp_async4(smem + L::XLT + j0 + 1, A.lamh + (ptrdiff_t)(a - 1) * g.W + c0 + j0 + 1);
    }
    if (last_row_here && (a + 1 < g.NR || g.cut_bot)) {
#pragma unroll
      for (int c = 0; c < 2; ++c) {
        cp_async4(smem + L::XPB + j0 + c, A.P1 + (size_t)(a * 128 + 128 + a) * g.W + c0 + j0 + c);
        cp_async4(smem + L::XLB + j0 + c, A.lamh + (size_t)a * g.W + c0 + j0 + c);
      }
    }
    if (tx == 0 && b > 0) {
#pragma unroll
      for (int r = 0; r < 4; ++r) cp_async4(smem + L::XLL + lr0 + r, A.lamv + (size_t)(b - 1) * g.H + gb + lr0 + r);
    }
    if (tx < 4 && b + 1 < g.NC) cp_async4(smem + L::XLR + lr0 + tx, A.lamv + (size_t)b * g.H + gb + lr0 + tx);
    if (need_qh) {
#pragma unroll
      for (int c = 0; c < 2; ++c) cp_async4(smem + L::XQH + j0 + c, A.P1 + (size_t)(gb + BAND + a) * g.W + c0 + j0 + c);
    }
    cp_async_commit();
  };

  bool timed_out = false;
  uint32_t phU = 0, phQ = 0;  // index of the next phase of mbU / mbQ this CTA waits for
  auto wait_u = [&]() {
    if (!mbar_wait(mbU, phU & 1)) timed_out = true;
    ++phU;
    if (tx == 0) mbar_arrive_expect_tx(mbU, kHaloBytes);  // arm the next phase
  };
  auto wait_q = [&]() {
    if (!mbar_wait(mbQ, phQ & 1)) timed_out = true;
    ++phQ;
    if (tx == 0) mbar_arrive_expect_tx(mbQ, kHaloBytes);
  };

  if (first < T) prefetch(first);

  for (int t = first; t < T; t += stride) {
    const int img = S.image(t);
    const LocalArgs& A = S.args(t);
    const Grid g = A.g;
    const int W2 = g.W + g.NC;
    const float tau = A.tau;
    const int lt = S.local(t);
    const int a = lt / g.NC, b = lt - a * g.NC;
    const int c0 = b * 128;
    const int gb = a * 128 + rank * BAND;
    const bool s_top = a > 0 || g.cut_top, s_bot = a + 1 < g.NR || g.cut_bot, s_lft = b > 0, s_rgt = b + 1 < g.NC;
    const float lim_left = (tx == 0 && !s_lft) ? 0.f : 1.f;
    const float lim_top = (i0 == 0 && !s_top) ? 0.f : 1.f;
    const bool right_lane = s_rgt && tx < 4;

    cp_async_wait_all();
    __syncthreads();  // staging landed; the previous subdomain's shared arrays are free
    if (img != cur_img) {  // made visible by the barrier after the unpack
      for (int q = tid; q < 8 * min(K, L::kMaxSmemCoef); q += NT) sCo[q] = reinterpret_cast<const float*>(A.coef)[q];
      cur_img = img;
    }
    auto tile_body = [&](auto fidc) {
    constexpr int FID = decltype(fidc)::value;
    // pairs [column c][e]: rows (e, e + 2) of column j0 + c
    f32x2 U[2][2], P1[2][2], P2[2][2], H1[2][2], H2[2][2], Q1[2][2], Q2[2][2];
    uint32_t in_d = 0;  // bit 4c + r: pixel (row r, column j0 + c) lies in the inpainting domain
    float pB[2] = {0.f, 0.f}, hB[2] = {0.f, 0.f};
    {
      float u[4][2], fv[4][2], p1[4][2], p2[4][2];
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        const float2 uu = *reinterpret_cast<const float2*>(smem + L::SU + (lr0 + r) * BW + j0);
        const float2 ff = *reinterpret_cast<const float2*>(smem + L::SU + BAND * BW + (lr0 + r) * BW + j0);
        const float2 q1 = *reinterpret_cast<const float2*>(smem + L::SU + 2 * BAND * BW + (lr0 + r) * BW + j0);
        const float2 q2 = *reinterpret_cast<const float2*>(smem + L::SP2 + (lr0 + r) * L::P2S + j0);
        u[r][0] = uu.x;
        u[r][1] = uu.y;
        fv[r][0] = ff.x;
        fv[r][1] = ff.y;
        p1[r][0] = q1.x;
        p1[r][1] = q1.y;
        p2[r][0] = q2.x;
        p2[r][1] = q2.y;
#pragma unroll
        for (int c = 0; c < 2; ++c) {
          if (FID == FID_SEG) fv[r][c] = (fv[r][c] - A.c1) * (fv[r][c] - A.c1) - (fv[r][c] - A.c2) * (fv[r][c] - A.c2);
          if (MASK && A.mask[(size_t)(gb + lr0 + r) * g.W + c0 + j0 + c]) in_d |= 1u << (4 * c + r);
        }
      }
      float h1[4][2], h2[4][2];
#pragma unroll
      for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int c = 0; c < 2; ++c) {
          h1[r][c] = p1[r][c];
          h2[r][c] = p2[r][c];
        }
      if (i0 == 0 && s_top) {
#pragma unroll
        for (int c = 0; c < 2; ++c) h1[0][c] = phat_t(p1[0][c], smem[L::XLT + j0 + c], tau);
      }
      if (tx == 0 && s_lft) {
#pragma unroll
        for (int r = 0; r < 4; ++r) h2[r][0] = phat_t(p2[r][0], smem[L::XLL + lr0 + r], tau);
      }
#pragma unroll
      for (int c = 0; c < 2; ++c)
#pragma unroll
        for (int e = 0; e < 2; ++e) {
          U[c][e] = pk2(u[e][c], u[e + 2][c]);
          P1[c][e] = pk2(p1[e][c], p1[e + 2][c]);
          P2[c][e] = pk2(p2[e][c], p2[e + 2][c]);
          H1[c][e] = pk2(h1[e][c], h1[e + 2][c]);
          H2[c][e] = pk2(h2[e][c], h2[e + 2][c]);
          Q1[c][e] = P1[c][e];
          Q2[c][e] = P2[c][e];
        }
#pragma unroll
      for (int c = 0; c < 2; ++c)
        *reinterpret_cast<ulonglong2*>(sF + ((ty * 2 + c) * NX + tx) * 4) =
            make_ulonglong2(pk2(fv[0][c], fv[2][c]), pk2(fv[1][c], fv[3][c]));
      *reinterpret_cast<ulonglong2*>(myQL) = make_ulonglong2(P2[0][0], P2[0][1]);
      *reinterpret_cast<float2*>(sQ1 + ty * BW + j0) = make_float2(p1[0][0], p1[0][1]);
      if (last_row_here) {
        if (s_bot) {
#pragma unroll
          for (int c = 0; c < 2; ++c) {
            pB[c] = smem[L::XPB + j0 + c];
            hB[c] = phat_s(pB[c], smem[L::XLB + j0 + c], tau);
          }
        }
        *reinterpret_cast<float2*>(sQ1 + TR * BW + j0) = make_float2(pB[0], pB[1]);
      }
      if (need_qh)
        *reinterpret_cast<float2*>(sQ1 + TR * BW + j0) = *reinterpret_cast<const float2*>(smem + L::XQH + j0);
      if (tx < 4) {
        const int lr = lr0 + tx;
        float pr = 0.f, hr = 0.f;
        if (s_rgt) {
          pr = smem[L::SP2 + lr * L::P2S + 128];
          hr = phat_s(pr, smem[L::XLR + lr], tau);
        }
        sPR[lr] = pr;
        sHR[lr] = hr;
        sQL[ty * L::SLOT + 4 * NX + (tx & 1) * 2 + (tx >> 1)] = pr;
      }
    }
    __syncthreads();  // staging consumed by every thread
    if (t + stride < T) prefetch(t + stride);

    for (int k = 0; k < K; ++k) {
      Coef co;
      if (k < L::kMaxSmemCoef) {
        const float4 ca = *reinterpret_cast<const float4*>(sCo + 8 * k);
        const float4 cb = *reinterpret_cast<const float4*>(sCo + 8 * k + 4);
        co = Coef{ca.x, ca.y, ca.z, ca.w, cb.x, cb.y, cb.z, cb.w};
      } else {
        co = A.coef[k];
      }
      const f32x2 SIG = pk2(co.sig, co.sig), UA = pk2(co.ua, co.ua), UB = pk2(co.ub, co.ub);
      const f32x2 PA = pk2(co.pa, co.pa), PC = pk2(co.pc, co.pc), PB = pk2(co.pb, co.pb), TH = pk2(co.th, co.th);
      if (need_qh && k > 0) wait_q();  // pbar1 halo of iteration k-1
      // ---- u-step: pair e = 1 (holding the thread's last row) first
      {
        const ulonglong2 qr = *reinterpret_cast<const ulonglong2*>(myQL + 4);  // left edge of the thread to the right
        const float2 qb = *reinterpret_cast<const float2*>(sQ1 + (ty + 1) * BW + j0);  // pbar1 of the row below
        const ulonglong2 fc0 = *reinterpret_cast<const ulonglong2*>(sF + ((ty * 2 + 0) * NX + tx) * 4);
        const ulonglong2 fc1 = *reinterpret_cast<const ulonglong2*>(sF + ((ty * 2 + 1) * NX + tx) * 4);
#pragma unroll
        for (int ee = 0; ee < 2; ++ee) {
          const int e = 1 - ee;
#pragma unroll
          for (int c = 0; c < 2; ++c) {
            const f32x2 below = e == 0 ? Q1[c][1] : pk2(hi2(Q1[c][0]), c == 0 ? qb.x : qb.y);
            const f32x2 right = c == 0 ? Q2[1][e] : (e == 0 ? qr.x : qr.y);
            const f32x2 d = sub2(add2(sub2(below, Q1[c][e]), right), Q2[c][e]);  // div_px
            const f32x2 fg = c == 0 ? (e == 0 ? fc0.x : fc0.y) : (e == 0 ? fc1.x : fc1.y);
            const f32x2 ub = fma2(SIG, d, U[c][e]);
            const bool dl = MASK && ((in_d >> (4 * c + e)) & 1u), dh = MASK && ((in_d >> (4 * c + e + 2)) & 1u);
            f32x2 un;
            if (FID == FID_L2) {
              un = fma2(UB, fg, mul2(UA, ub));
              if (MASK) un = pk2(dl ? lo2(ub) : lo2(un), dh ? hi2(ub) : hi2(un));
            } else {
              un = pk2(prox_ubar<FID>(lo2(ub), lo2(fg), dl, co), prox_ubar<FID>(hi2(ub), hi2(fg), dh, co));
            }
            U[c][e] = un;
          }
          if (e == 1 && push_down) st_async_v2(remote_u, hi2(U[0][1]), hi2(U[1][1]), remote_mbU);
        }
        *reinterpret_cast<ulonglong2*>(myUR) = make_ulonglong2(U[1][0], U[1][1]);
        if (ty < TR - 1) *reinterpret_cast<float2*>(sUB + (ty + 1) * BW + j0) = make_float2(hi2(U[0][1]), hi2(U[1][1]));
      }
      __syncthreads();
      if (need_uh) wait_u();  // u halo of iteration k
      // ---- p-step: pair e = 0 (holding the thread's first row) first
      {
        const float2 ua = *reinterpret_cast<const float2*>(sUB + ty * BW + j0);  // u of the row above
        const ulonglong2 ul = *reinterpret_cast<const ulonglong2*>(myUR - 4);    // right column of the thread to the left
#pragma unroll
        for (int e = 0; e < 2; ++e) {
#pragma unroll
          for (int c = 0; c < 2; ++c) {
            const f32x2 above = e == 1 ? U[c][0] : pk2(c == 0 ? ua.x : ua.y, lo2(U[c][1]));
            const f32x2 leftu = c == 1 ? U[0][e] : (e == 0 ? ul.x : ul.y);
            {
              const f32x2 tt = fma2(PC, sub2(U[c][e], above), fma2(PA, P1[c][e], mul2(PB, H1[c][e])));  // p_target
              const float l0 = e == 0 ? lim_top : 1.f;
              const f32x2 pn = pk2(clamp_abs(lo2(tt), l0), clamp_abs(hi2(tt), 1.f));
              Q1[c][e] = fma2(TH, sub2(pn, P1[c][e]), pn);
              P1[c][e] = pn;
            }
            {
              const f32x2 tt = fma2(PC, sub2(U[c][e], leftu), fma2(PA, P2[c][e], mul2(PB, H2[c][e])));
              const float l = c == 0 ? lim_left : 1.f;
              const f32x2 pn = pk2(clamp_abs(lo2(tt), l), clamp_abs(hi2(tt), l));
              Q2[c][e] = fma2(TH, sub2(pn, P2[c][e]), pn);
              P2[c][e] = pn;
            }
          }
          if (e == 0) {
            const float qa = lo2(Q1[0][0]), qc = lo2(Q1[1][0]);
            if (ty > 0) *reinterpret_cast<float2*>(sQ1 + ty * BW + j0) = make_float2(qa, qc);
            if (push_up) st_async_v2(remote_q1, qa, qc, remote_mbQ);
          }
        }
        *reinterpret_cast<ulonglong2*>(myQL) = make_ulonglong2(Q2[0][0], Q2[0][1]);
      }
      if (last_row_here && s_bot) {
#pragma unroll
        for (int c = 0; c < 2; ++c) {
          float qB;
          p_update(pB[c], qB, -hi2(U[c][1]), hB[c], co);
          sQ1[TR * BW + j0 + c] = qB;
        }
      }
      if (right_lane) {
        const int lr = lr0 + tx;
        const int pos = (tx & 1) * 2 + (tx >> 1);
        float pr = sPR[lr], qr;
        p_update(pr, qr, -sUR[ty * L::SLOT + 4 * NX + pos], sHR[lr], co);
        sPR[lr] = pr;
        sQL[ty * L::SLOT + 4 * NX + pos] = qr;
      }
      __syncthreads();
    }
    if (need_qh) wait_q();  // drain the last pbar1 halo (not read)

#pragma unroll
    for (int r = 0; r < 4; ++r) {
      const int e = r & 1, h = r >> 1;
      const int gi = gb + lr0 + r;
      *reinterpret_cast<float2*>(A.u + (size_t)gi * g.W + c0 + j0) = make_float2(lane_of(U[0][e], h), lane_of(U[1][e], h));
      *reinterpret_cast<float2*>(A.P1 + (size_t)(gi + a) * g.W + c0 + j0) =
          make_float2(lane_of(P1[0][e], h), lane_of(P1[1][e], h));
      float* p2row = A.P2 + (size_t)gi * W2 + c0 + b + j0;
      p2row[0] = lane_of(P2[0][e], h);
      p2row[1] = lane_of(P2[1][e], h);
    }
    const Strips out = S.out(t);
    if (i0 == 0 && s_top) {
      out.ST[(ptrdiff_t)(a - 1) * g.W + c0 + j0] = lo2(P1[0][0]);
      out.ST[(ptrdiff_t)(a - 1) * g.W + c0 + j0 + 1] = lo2(P1[1][0]);
    }
    if (tx == 0 && s_lft) {
#pragma unroll
      for (int r = 0; r < 4; ++r) out.SL[(size_t)(b - 1) * g.H + gb + lr0 + r] = lane_of(P2[0][r & 1], r >> 1);
    }
    if (last_row_here && s_bot) {
#pragma unroll
      for (int c = 0; c < 2; ++c) {
        A.P1[(size_t)(a * 128 + 128 + a) * g.W + c0 + j0 + c] = pB[c];
        out.SB[(size_t)a * g.W + c0 + j0 + c] = pB[c];
      }
    }
    if (right_lane) {
      const int gi = gb + lr0 + tx;
      const float pr = sPR[lr0 + tx];
      A.P2[(size_t)gi * W2 + c0 + 128 + b] = pr;
      out.SR[(size_t)b * g.H + gi] = pr;
    }
    };  // tile_body
    S.dispatch(t, tile_body);
  }
  cp_async_wait_all();
  cluster_arrive<true>();  // no CTA leaves while a neighbour may still write into it
  cluster_wait();
  if (timed_out) atomicOr(S.err(), 1);
}

template <int FID, bool MASK>
__global__ void __launch_bounds__(MtLayout::NT, 2) k_fused_mt(const LocalArgs A) {
  fused_mt_body<FID, MASK>(A, blockIdx.y, gridDim.y);
}

// Persistent kernel over the work list of a batch: cluster c runs tiles c, c + C, ...
// of the batch, each with its image's fidelity, parameters and coefficients.
__global__ void __launch_bounds__(MtLayout::NT, 2) k_fused_mt_batch(const BatchArgs B, int total) {
  fused_mt_run<false>(BatchTiles{B, total}, blockIdx.y, gridDim.y);
}

template <int FID, bool MASK>
int& mt_clusters(int dev) {
  static int n[64] = {0};
  return n[dev & 63];
}

cudaLaunchConfig_t mt_config(int clusters, cudaLaunchAttribute* attr) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(MtLayout::CL, clusters, 1);
  cfg.blockDim = dim3(MtLayout::NX, MtLayout::TR, 1);
  cfg.dynamicSmemBytes = MtLayout::BYTES;
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = MtLayout::CL;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cfg;
}

template <int FID, bool MASK>
cudaError_t prepare_mt_one() {
  auto kern = k_fused_mt<FID, MASK>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)MtLayout::BYTES);
  if (e != cudaSuccess) return e;
  cudaLaunchAttribute attr[1];
  cudaLaunchConfig_t cfg = mt_config(1024, attr);
  int n = 0;
  if (cudaOccupancyMaxActiveClusters(&n, kern, &cfg) != cudaSuccess) {
    cudaGetLastError();
    n = 0;
  }
  int dev = 0;
  cudaGetDevice(&dev);
  mt_clusters<FID, MASK>(dev) = n;
  return cudaSuccess;
}

template <int FID, bool MASK>
cudaError_t launch_mt_one(const LocalArgs& a, cudaStream_t st) {
  int dev = 0;
  cudaGetDevice(&dev);
  const int tiles = a.g.NR * a.g.NC;
  int nc = mt_clusters<FID, MASK>(dev);
  if (nc <= 0 || nc > tiles) nc = tiles;
  cudaLaunchAttribute attr[1];
  cudaLaunchConfig_t cfg = mt_config(nc, attr);
  cfg.stream = st;
  return cudaLaunchKernelEx(&cfg, k_fused_mt<FID, MASK>, a);
}

int& mt_batch_clusters(int dev) {
  static int n[64] = {0};
  return n[dev & 63];
}

}  // namespace

cudaError_t fused_mt_batch_prepare() {
  cudaError_t e =
      cudaFuncSetAttribute(k_fused_mt_batch, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)MtLayout::BYTES);
  if (e != cudaSuccess) return e;
  cudaLaunchAttribute attr[1];
  cudaLaunchConfig_t cfg = mt_config(1024, attr);
  int n = 0;
  if (cudaOccupancyMaxActiveClusters(&n, k_fused_mt_batch, &cfg) != cudaSuccess) {
    cudaGetLastError();
    n = 0;
  }
  int dev = 0;
  cudaGetDevice(&dev);
  mt_batch_clusters(dev) = n;
  return cudaSuccess;
}

cudaError_t launch_fused_mt_batch(const BatchArgs& B, int total_tiles, cudaStream_t st) {
  int dev = 0;
  cudaGetDevice(&dev);
  int nc = mt_batch_clusters(dev);
  if (nc <= 0 || nc > total_tiles) nc = total_tiles;
  cudaLaunchAttribute attr[1];
  cudaLaunchConfig_t cfg = mt_config(nc, attr);
  cfg.stream = st;
  return cudaLaunchKernelEx(&cfg, k_fused_mt_batch, B, total_tiles);
}

bool fused_mt_supported(const LocalArgs& a) {
  auto al16 = [](const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15) == 0; };
  return a.g.H == 128 * a.g.NR && a.g.W == 128 * a.g.NC && al16(a.u) && al16(a.f) && al16(a.P1);
}

cudaError_t fused_mt_prepare() {
  cudaError_t e;
  if ((e = prepare_mt_one<FID_L2, false>()) != cudaSuccess) return e;
  if ((e = prepare_mt_one<FID_L2, true>()) != cudaSuccess) return e;
  if ((e = prepare_mt_one<FID_L1, false>()) != cudaSuccess) return e;
  if ((e = prepare_mt_one<FID_L1, true>()) != cudaSuccess) return e;
  if ((e = prepare_mt_one<FID_SEG, false>()) != cudaSuccess) return e;
  return fused_mt_batch_prepare();
}

cudaError_t launch_fused_mt(const LocalArgs& a, int fid, cudaStream_t st) {
  const bool m = a.mask != nullptr;
  switch (fid) {
    case FID_L2: return m ? launch_mt_one<FID_L2, true>(a, st) : launch_mt_one<FID_L2, false>(a, st);
    case FID_L1: return m ? launch_mt_one<FID_L1, true>(a, st) : launch_mt_one<FID_L1, false>(a, st);
    default: return launch_mt_one<FID_SEG, false>(a, st);
  }
}

}  // namespace ddtv
