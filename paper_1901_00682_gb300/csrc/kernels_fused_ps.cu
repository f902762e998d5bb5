// Persistent fused local solver: the column mapping of fused_pa_body with 16-byte
// state copies and an out-buffer.
//
// Same on-chip mapping and inner loop as fused_pa_body with packed row pairs (r, r +
// R/2), so the results are bit-identical; only the movement of the state between
// subdomains differs:
//   * the next subdomain's state is prefetched by 16-byte cp.async copies into
//     row-major staging arrays (p2 is fetched as a 132-float window that starts on a
//     16-byte boundary, which needs W + N_c to be a multiple of 4; f goes straight
//     into the second half of a double-buffered f array that the inner loop reads, so
//     it is never copied again);
//   * the results of a subdomain go to an out-buffer in shared memory at the switch
//     (conflict-free stores) and are written back with 16-byte stores for u and p1,
//     whose rows are 16-byte aligned, right after the next subdomain's unpack.
// The out-buffer is rewritten only at the next switch, after the CTA barrier that
// ends every inner iteration; the staging arrays are refilled only after the unpack of
// the subdomain they hold.
#include "fused_common.cuh"
#include "internal.cuh"

namespace ddtv {

namespace {

struct PsLayout {
  static constexpr int R = 8, TR = 2, CL = 8, BW = 128, BAND = R * TR, NT = BW * TR;
  static constexpr int US = BW + 1, QS = BW + 1, P2S = 132;
  static constexpr int U = 0;                           // (BAND + 1) x US: row 0 = u above the band; index 0 = zero pad
  static constexpr int Q2 = U + (BAND + 1) * US;        // BAND x QS: pbar2; index 128 = right side
  static constexpr int Q1 = Q2 + BAND * QS;             // (TR + 1) x BW: first-row pbar1 per thread row; row TR = below
  static constexpr int PR = Q1 + (TR + 1) * BW;         // BAND right-side p
  static constexpr int HR = PR + BAND;                  // BAND right-side phat
  static constexpr int CO = (HR + BAND + 3) & ~3;       // kMaxSmemCoef x 8 coefficients
  static constexpr int kMaxSmemCoef = 64;
  static constexpr int F = CO + 16 * kMaxSmemCoef;      // 2 x BAND x BW: f (or g) of this and of the next subdomain
  static constexpr int SU = F + 2 * BAND * BW;          // staging: u (BAND x BW)
  static constexpr int SP1 = SU + BAND * BW;            // p1 (BAND x BW)
  static constexpr int SP2 = SP1 + BAND * BW;           // p2 window (BAND x P2S)
  static constexpr int XLT = SP2 + BAND * P2S;          // lamh above the tile (BW)
  static constexpr int XPB = XLT + BW;                  // p1 of the tile's bottom side (BW)
  static constexpr int XLB = XPB + BW;                  // lamh below the tile (BW)
  static constexpr int XQH = XLB + BW;                  // p1 of the first row below the band (BW)
  static constexpr int XLL = XQH + BW;                  // lamv left of the band (BAND)
  static constexpr int XLR = XLL + BAND;                // lamv right of the band (BAND)
  static constexpr int OU = XLR + BAND;                 // out-buffer: u (BAND x BW)
  static constexpr int OP1 = OU + BAND * BW;            // p1 (BAND x BW)
  static constexpr int OP2 = OP1 + BAND * BW;           // p2, columns 0..128 of the tile (BAND x P2S)
  static constexpr int MB = OP2 + BAND * P2S;           // two mbarriers
  static constexpr size_t BYTES = sizeof(float) * MB + 16;
  static constexpr int kPre = 10;                       // copies per thread and subdomain
  static constexpr int kOut = 13;                       // stores per thread and subdomain
  static_assert(CO % 4 == 0 && F % 4 == 0 && SU % 4 == 0 && SP1 % 4 == 0 && SP2 % 4 == 0 && XLT % 4 == 0 &&
                    XLL % 4 == 0 && XLR % 4 == 0 && OU % 4 == 0 && OP1 % 4 == 0 && MB % 2 == 0,
                "16-byte alignment of the vector and cp.async buffers");
  static_assert(CL * BAND == 128, "a cluster of CTAs covers the 128 rows of a tile");
};

template <int FID, bool MASK>
__device__ __forceinline__ void fused_ps_body(const LocalArgs& A, const int first, const int stride) {
  using L = PsLayout;
  constexpr int R = L::R, TR = L::TR, CL = L::CL, BW = L::BW, BAND = L::BAND, NT = L::NT, H2 = R / 2;
  extern __shared__ __align__(16) float smem[];
  float* sU = smem + L::U;
  float* sQ2 = smem + L::Q2;
  float* sQ1 = smem + L::Q1;
  float* sPR = smem + L::PR;
  float* sHR = smem + L::HR;
  float* sCo = smem + L::CO;
  const uint32_t mbU = smem_addr(smem + L::MB);
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
  const bool need_uh = push_up;
  const bool need_qh = push_down;
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
  if (need_uh && j == 0) mbar_arrive_expect_tx(mbU, kHaloBytes);
  if (need_qh && j == 0) mbar_arrive_expect_tx(mbQ, kHaloBytes);
  cluster_arrive<true>();  // barriers initialised and armed everywhere before any halo is sent
  cluster_wait();

  // copy m of the prefetch of tile (a, b) into the staging arrays (f into F[fbuf])
  auto pre_slot = [&](int m, int a, int b, int fbuf) {
    const int c0 = b * 128, gb = a * 128 + rank * BAND;
    if (m < 6) {  // u, f, p1: BAND rows x 32 chunks of 16 bytes, two chunks per thread each
      const int fld = m >> 1, q = tid + NT * (m & 1), row = q >> 5, ch = q & 31;
      if (fld == 0) cp_async16(smem + L::SU + row * BW + 4 * ch, A.u + (size_t)(gb + row) * g.W + c0 + 4 * ch);
      if (fld == 1)
        cp_async16(smem + L::F + fbuf * BAND * BW + row * BW + 4 * ch, A.f + (size_t)(gb + row) * g.W + c0 + 4 * ch);
      if (fld == 2)
        cp_async16(smem + L::SP1 + row * BW + 4 * ch, A.P1 + (size_t)(gb + row + a) * g.W + c0 + 4 * ch);
    } else if (m < 9) {  // p2 window: BAND rows x 33 chunks
      const int q = tid + NT * (m - 6);
      if (q < BAND * 33) {
        const int row = q / 33, ch = q - row * 33;
        cp_async16(smem + L::SP2 + row * L::P2S + 4 * ch, A.P2 + (size_t)(gb + row) * W2 + c0 + b - (b & 3) + 4 * ch);
      }
    } else {  // the multipliers and neighbouring rows of the sides
      if (tid < 32) {
        if (rank == 0 && a > 0) cp_async16(smem + L::XLT + 4 * tid, A.lamh + (size_t)(a - 1) * g.W + c0 + 4 * tid);
      } else if (tid < 64) {
        if (rank == CL - 1 && a + 1 < g.NR)
          cp_async16(smem + L::XPB + 4 * (tid - 32), A.P1 + (size_t)(a * 128 + 128 + a) * g.W + c0 + 4 * (tid - 32));
      } else if (tid < 96) {
        if (rank == CL - 1 && a + 1 < g.NR)
          cp_async16(smem + L::XLB + 4 * (tid - 64), A.lamh + (size_t)a * g.W + c0 + 4 * (tid - 64));
      } else if (tid < 128) {
        if (rank < CL - 1) cp_async16(smem + L::XQH + 4 * (tid - 96), A.P1 + (size_t)(gb + BAND + a) * g.W + c0 + 4 * (tid - 96));
      } else if (tid < 132) {
        if (b > 0) cp_async16(smem + L::XLL + 4 * (tid - 128), A.lamv + (size_t)(b - 1) * g.H + gb + 4 * (tid - 128));
      } else if (tid < 136) {
        if (b + 1 < g.NC) cp_async16(smem + L::XLR + 4 * (tid - 132), A.lamv + (size_t)b * g.H + gb + 4 * (tid - 132));
      }
    }
  };
  // store m of the out-buffer, which holds tile (a, b)
  auto out_slot = [&](int m, int a, int b) {
    const int c0 = b * 128, gb = a * 128 + rank * BAND;
    if (m < 4) {  // u, p1: BAND rows x 32 chunks of 16 bytes, two chunks per thread each
      const int q = tid + NT * (m & 1), row = q >> 5, ch = q & 31;
      if (m < 2)
        *reinterpret_cast<float4*>(A.u + (size_t)(gb + row) * g.W + c0 + 4 * ch) =
            *reinterpret_cast<const float4*>(smem + L::OU + row * BW + 4 * ch);
      else
        *reinterpret_cast<float4*>(A.P1 + (size_t)(gb + row + a) * g.W + c0 + 4 * ch) =
            *reinterpret_cast<const float4*>(smem + L::OP1 + row * BW + 4 * ch);
    } else {  // p2: BAND rows x 129 values (the window is not 16-byte aligned)
      const int q = tid + NT * (m - 4);
      if (q < BAND * 129) {
        const int row = q / 129, col = q - row * 129;
        A.P2[(size_t)(gb + row) * W2 + c0 + b + col] = smem[L::OP2 + row * L::P2S + col];
      }
    }
  };

  bool timed_out = false;
  uint32_t phU = 0, phQ = 0;
  auto wait_u = [&]() {
    if (!mbar_wait(mbU, phU & 1)) timed_out = true;
    ++phU;
    if (j == 0) mbar_arrive_expect_tx(mbU, kHaloBytes);
  };
  auto wait_q = [&]() {
    if (!mbar_wait(mbQ, phQ & 1)) timed_out = true;
    ++phQ;
    if (j == 0) mbar_arrive_expect_tx(mbQ, kHaloBytes);
  };

  float* sUr = sU + (lr0 + 1) * L::US + j + 1;
  float* sQ2r = sQ2 + lr0 * L::QS + j;
  if (first < T) {
    for (int m = 0; m < L::kPre; ++m) pre_slot(m, first / g.NC, first % g.NC, 0);
    cp_async_commit();
  }
  int prev = -1, pa = 0, pb = 0;  // tile held by the out-buffer (-1: none) and its grid position
  uint32_t nsub = 0;

  for (int t = first; t < T; t += stride, ++nsub) {
    const int a = t / g.NC, b = t - a * g.NC;
    const int c0 = b * 128, gj = c0 + j, gb = a * 128 + rank * BAND;
    const bool s_top = a > 0, s_bot = a + 1 < g.NR, s_lft = b > 0, s_rgt = b + 1 < g.NC;
    const float lim_left = (j == 0 && !s_lft) ? 0.f : 1.f;
    const float lim_top = (i0 == 0 && !s_top) ? 0.f : 1.f;
    const bool right_lane = s_rgt && j < R;
    const int o = b & 3;
    const int cur = nsub & 1;
    float* sFc = smem + L::F + cur * BAND * BW;
    const float* sFr = sFc + lr0 * BW + j;
    const int tn = t + stride < T ? t + stride : -1;  // tile prefetched while this one iterates
    const int na = tn / g.NC, nb = tn - na * g.NC;
    f32x2 U[H2], P1v[H2], P2v[H2], H1v[H2], H2v[H2], Q1v[H2];
    uint32_t in_d = 0;
    float pB = 0.f, hB = 0.f;

    cp_async_wait_all();
    __syncthreads();  // staging landed; the previous subdomain's shared arrays are free
    {
      float u[R], p1[R], p2[R], h1[R], h2[R];
#pragma unroll
      for (int r = 0; r < R; ++r) {
        const int lr = lr0 + r;
        u[r] = smem[L::SU + lr * BW + j];
        if (FID == FID_SEG) {
          const float fv = sFc[lr * BW + j];
          sFc[lr * BW + j] = (fv - A.c1) * (fv - A.c1) - (fv - A.c2) * (fv - A.c2);
        }
        if (MASK && A.mask[(size_t)(gb + lr) * g.W + gj]) in_d |= 1u << r;
        p1[r] = smem[L::SP1 + lr * BW + j];
        p2[r] = smem[L::SP2 + lr * L::P2S + o + j];
        h1[r] = p1[r];
        h2[r] = p2[r];
        sQ2[lr * L::QS + j] = p2[r];
        sU[(lr + 1) * L::US] = 0.f;
      }
      if (i0 == 0 && s_top) h1[0] = phat_t(p1[0], smem[L::XLT + j], tau);
      if (j == 0 && s_lft) {
#pragma unroll
        for (int r = 0; r < R; ++r) h2[r] = phat_t(p2[r], smem[L::XLL + lr0 + r], tau);
      }
      if (last_row_here) {
        if (s_bot) {
          pB = smem[L::XPB + j];
          hB = phat_s(pB, smem[L::XLB + j], tau);
        }
        sQ1[TR * BW + j] = pB;
      }
      if (need_qh) sQ1[TR * BW + j] = smem[L::XQH + j];  // first row of the band below
      if (j < R) {
        const int lr = lr0 + j;
        float pr = 0.f, hr = 0.f;
        if (s_rgt) {
          pr = smem[L::SP2 + lr * L::P2S + o + 128];
          hr = phat_s(pr, smem[L::XLR + lr], tau);
        }
        sPR[lr] = pr;
        sHR[lr] = hr;
        sQ2[lr * L::QS + 128] = pr;
      }
      sQ1[ty * BW + j] = p1[0];
#pragma unroll
      for (int i = 0; i < H2; ++i) {
        U[i] = pk2(u[i], u[i + H2]);
        P1v[i] = pk2(p1[i], p1[i + H2]);
        P2v[i] = pk2(p2[i], p2[i + H2]);
        H1v[i] = pk2(h1[i], h1[i + H2]);
        H2v[i] = pk2(h2[i], h2[i + H2]);
        Q1v[i] = P1v[i];
      }
    }
    __syncthreads();  // staging consumed by every thread
    if (tn >= 0) {
      for (int m = 0; m < L::kPre; ++m) pre_slot(m, na, nb, cur ^ 1);
      cp_async_commit();
    }
    if (prev >= 0)
      for (int m = 0; m < L::kOut; ++m) out_slot(m, pa, pb);

    for (int k = 0; k < K; ++k) {
      // a share of the state traffic: the next tile's copies, the previous tile's stores
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
          const f32x2 pn =
              pk2(fminf(fmaxf(lo2(tt), -lim_left), lim_left), fminf(fmaxf(hi2(tt), -lim_left), lim_left));
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
    if (need_qh) wait_q();  // drain the last pbar1 halo (not read)

    // results into the out-buffer (written back during the next tile's iterations);
    // the sides' strips and the bottom side directly
#pragma unroll
    for (int i = 0; i < H2; ++i) {
      smem[L::OU + (lr0 + i) * BW + j] = lo2(U[i]);
      smem[L::OU + (lr0 + i + H2) * BW + j] = hi2(U[i]);
      smem[L::OP1 + (lr0 + i) * BW + j] = lo2(P1v[i]);
      smem[L::OP1 + (lr0 + i + H2) * BW + j] = hi2(P1v[i]);
      smem[L::OP2 + (lr0 + i) * L::P2S + j] = lo2(P2v[i]);
      smem[L::OP2 + (lr0 + i + H2) * L::P2S + j] = hi2(P2v[i]);
    }
    if (j < R) smem[L::OP2 + (lr0 + j) * L::P2S + 128] = sPR[lr0 + j];  // right side (0 on the image boundary)
    if (i0 == 0 && s_top) A.out.ST[(size_t)(a - 1) * g.W + gj] = lo2(P1v[0]);
    if (j == 0 && s_lft) {
#pragma unroll
      for (int i = 0; i < H2; ++i) {
        A.out.SL[(size_t)(b - 1) * g.H + gb + lr0 + i] = lo2(P2v[i]);
        A.out.SL[(size_t)(b - 1) * g.H + gb + lr0 + i + H2] = hi2(P2v[i]);
      }
    }
    if (last_row_here && s_bot) {
      A.P1[(size_t)(a * 128 + 128 + a) * g.W + gj] = pB;
      A.out.SB[(size_t)a * g.W + gj] = pB;
    }
    if (right_lane) A.out.SR[(size_t)b * g.H + gb + lr0 + j] = sPR[lr0 + j];
    prev = t;
    pa = a;
    pb = b;
  }
  if (prev >= 0) {  // the last tile's results
    __syncthreads();
    for (int m = 0; m < L::kOut; ++m) out_slot(m, pa, pb);
  }
  cp_async_wait_all();
  cluster_arrive<true>();  // no CTA leaves while a neighbour may still write into it
  cluster_wait();
  if (timed_out) atomicOr(A.err, 1);
}

template <int FID, bool MASK>
__global__ void __launch_bounds__(PsLayout::NT, 2) k_fused_ps(const LocalArgs A) {
  fused_ps_body<FID, MASK>(A, blockIdx.y, gridDim.y);
}

template <int FID, bool MASK>
int& ps_clusters(int dev) {
  static int n[64] = {0};
  return n[dev & 63];
}

cudaLaunchConfig_t ps_config(int clusters, cudaLaunchAttribute* attr) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(PsLayout::CL, clusters, 1);
  cfg.blockDim = dim3(PsLayout::BW, PsLayout::TR, 1);
  cfg.dynamicSmemBytes = PsLayout::BYTES;
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = PsLayout::CL;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cfg;
}

template <int FID, bool MASK>
cudaError_t prepare_ps_one() {
  auto kern = k_fused_ps<FID, MASK>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)PsLayout::BYTES);
  if (e != cudaSuccess) return e;
  cudaLaunchAttribute attr[1];
  cudaLaunchConfig_t cfg = ps_config(1024, attr);
  int n = 0;
  if (cudaOccupancyMaxActiveClusters(&n, kern, &cfg) != cudaSuccess) {
    cudaGetLastError();
    n = 0;
  }
  int dev = 0;
  cudaGetDevice(&dev);
  ps_clusters<FID, MASK>(dev) = n;
  return cudaSuccess;
}

template <int FID, bool MASK>
cudaError_t launch_ps_one(const LocalArgs& a, cudaStream_t st) {
  int dev = 0;
  cudaGetDevice(&dev);
  const int tiles = a.g.NR * a.g.NC;
  int nc = ps_clusters<FID, MASK>(dev);
  if (nc <= 0 || nc > tiles) nc = tiles;
  cudaLaunchAttribute attr[1];
  cudaLaunchConfig_t cfg = ps_config(nc, attr);
  cfg.stream = st;
  return cudaLaunchKernelEx(&cfg, k_fused_ps<FID, MASK>, a);
}

}  // namespace

bool fused_ps_supported(const LocalArgs& a) {
  auto al16 = [](const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15) == 0; };
  return a.g.H == 128 * a.g.NR && a.g.W == 128 * a.g.NC && (a.g.W + a.g.NC) % 4 == 0 && al16(a.u) && al16(a.f) &&
         al16(a.P1) && al16(a.P2) && al16(a.lamh) && al16(a.lamv);
}

cudaError_t fused_ps_prepare() {
  cudaError_t e;
  if ((e = prepare_ps_one<FID_L2, false>()) != cudaSuccess) return e;
  if ((e = prepare_ps_one<FID_L2, true>()) != cudaSuccess) return e;
  if ((e = prepare_ps_one<FID_L1, false>()) != cudaSuccess) return e;
  if ((e = prepare_ps_one<FID_L1, true>()) != cudaSuccess) return e;
  return prepare_ps_one<FID_SEG, false>();
}

cudaError_t launch_fused_ps(const LocalArgs& a, int fid, cudaStream_t st) {
  const bool m = a.mask != nullptr;
  switch (fid) {
    case FID_L2: return m ? launch_ps_one<FID_L2, true>(a, st) : launch_ps_one<FID_L2, false>(a, st);
    case FID_L1: return m ? launch_ps_one<FID_L1, true>(a, st) : launch_ps_one<FID_L1, false>(a, st);
    default: return launch_ps_one<FID_SEG, false>(a, st);
  }
}

}  // namespace ddtv
