// Persistent fused local solver with one warp per pair of rows (128 x 128 subdomains).
//
// In the column mappings (kernels_fused.cu, kernels_fused_mt.cu) every inner iteration
// ends each half-step with a barrier over the whole CTA: a warp that waits for a halo
// row (or does the extra work of a subdomain side) holds up all the others.  Here a
// warp owns two full rows of the CTA's band, each lane a micro-tile of four columns by
// two rows, so
//   * horizontal neighbours are in the lane's registers or one shuffle away (the u of
//     the column to the left, the pbar2 of the edge to the right),
//   * the tile's right side (the p2 dofs of column 128) belongs to lane 31 and its
//     bottom side (the p1 dofs of row 128) to the last warp of the last CTA, both in
//     registers,
//   * only vertical neighbours cross warps: the u of a warp's last row (read by the
//     warp below for its p1 step) and the pbar1 of its first row (read by the warp
//     above for its u-step).  Each of these is one vector store, one named-barrier
//     arrive by the producing warp and one named-barrier sync by the consuming warp
//     (barrier IDs 1-7 for u, 8-14 for pbar1; the buffers are double-buffered by the
//     iteration's parity), so a warp waits only for the data it reads.
// Between the CTAs of a cluster the first and last rows travel with st.async and
// mbarrier complete_tx exactly as in fused_pa_body (same phase protocol, bounded
// waits, the last pbar1 halo of a subdomain drained).
//
// Arrival counts: barrier U(w) (w = 0..6) gets one arrive from warp w in every u-step
// and one sync from warp w + 1 in every p-step; barrier Q(w) (w = 1..7) gets one
// arrive from warp w in the p-steps 0..K-2 and one sync from warp w - 1 in the
// u-steps 1..K-1.  A producer cannot arrive twice before its consumer synced once:
// warp w's next u-step waits (Q(w + 1)) for data that warp w + 1 produces after its
// sync on U(w), and warp w's next p-step waits (U(w - 1)) for data that warp w - 1
// produces after its sync on Q(w).  All conditions on these instructions are uniform
// over a warp, and every warp passes a CTA barrier between subdomains.
//
// The next subdomain's u, f, p1 and p2 rows (and the multipliers of its sides) are
// prefetched with bulk asynchronous copies (cp.async.bulk, completion counted on an
// mbarrier); u and p1 are written back from shared memory with bulk copies as well,
// so neither the loads nor most of the stores hold up the warps.  This needs every
// row of u, f, p1 and p2 to start on a 16-byte boundary (W + N_c a multiple of 4);
// the p2 window of a tile is widened to 16-byte boundaries and indexed from its
// offset.  Rows are packed in pairs of columns (c, c + 2) for the `*.f32x2`
// arithmetic; every value is computed with the operations of the scalar iteration in
// the same order (pointwise.cuh), so the results are bit-identical to the other
// mappings.
#include "fused_common.cuh"
#include "internal.cuh"

namespace ddtv {

namespace {

struct WrLayout2 {
  static constexpr int CL = 8, NW = 8, BAND = 2 * NW, BW = 128, NT = 32 * NW;
  static constexpr int P2S = 132;                   // staged p2 row: 132 floats from a 16-byte boundary
  static constexpr int UBUF = 0;                    // [NW][2][128]: u of warp w's last row, by parity (pair order)
  static constexpr int QBUF = UBUF + NW * 2 * BW;   // [NW][2][128]: pbar1 of warp w's first row, by parity
  static constexpr int UH = QBUF + NW * 2 * BW;     // [128] u of the row above the band (halo; zero in CTA 0)
  static constexpr int QH = UH + BW;                // [128] pbar1 of the row below the band (halo)
  static constexpr int F = QH + BW;                 // [NW][32][2][4] f (or g) per lane and row, pair order
  static constexpr int CO = F + NW * 32 * 8;        // [kMaxSmemCoef][8] coefficients
  static constexpr int kMaxSmemCoef = 64;
  static constexpr int SU = CO + 16 * kMaxSmemCoef; // staging of the next subdomain: u, f, p1 [BAND][128] each
  static constexpr int SP2 = SU + 3 * BAND * BW;    // p2 [BAND][P2S]
  static constexpr int XLT = SP2 + BAND * P2S;      // lamh above the tile [128]
  static constexpr int XPB = XLT + BW;              // p1 of the tile's bottom side [128]
  static constexpr int XLB = XPB + BW;              // lamh below the tile [128]
  static constexpr int XQH = XLB + BW;              // p1 of the first row below the band [128]
  static constexpr int XLL = XQH + BW;              // lamv left of the band [BAND]
  static constexpr int XLR = XLL + BAND;            // lamv right of the band [BAND]
  static constexpr int SOU = XLR + BAND;            // outgoing u [BAND][128]
  static constexpr int SOP = SOU + BAND * BW;       // outgoing p1 [BAND][128]
  static constexpr int MB = SOP + BAND * BW;        // mbarriers: u halo, pbar1 halo, staging
  static constexpr size_t BYTES = sizeof(float) * MB + 32;
  static_assert(F % 4 == 0 && CO % 4 == 0 && SU % 4 == 0 && SP2 % 4 == 0 && XLT % 4 == 0 && XLL % 4 == 0 &&
                    XLR % 4 == 0 && SOU % 4 == 0 && MB % 4 == 0 && (P2S * 4) % 16 == 0,
                "16-byte alignment of vector and bulk-copy buffers");
  static_assert(CL * BAND == 128, "a cluster of CTAs covers the 128 rows of a tile");
};

__device__ __forceinline__ void bar_sync_n(int id, int n) { asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(n) : "memory"); }
__device__ __forceinline__ void bar_arrive_n(int id, int n) {
  asm volatile("bar.arrive %0, %1;" ::"r"(id), "r"(n) : "memory");
}

// bulk copy global -> own shared memory, counted on a local mbarrier
__device__ __forceinline__ void bulk_g2s(float* dst, const float* src, uint32_t bytes, uint32_t mbar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_addr(dst)),
               "l"(src), "r"(bytes), "r"(mbar)
               : "memory");
}
// bulk copy own shared memory -> global (bulk group of the issuing thread)
__device__ __forceinline__ void bulk_s2g(float* dst, const float* src, uint32_t bytes) {
  asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(dst), "r"(smem_addr(src)),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_read() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ void st_async_v4(uint32_t remote_addr, float a, float b, float c, float d,
                                            uint32_t remote_mbar) {
  asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.v4.b32 [%0], {%1, %2, %3, %4}, [%5];" ::"r"(
                   remote_addr),
               "r"(__float_as_uint(a)), "r"(__float_as_uint(b)), "r"(__float_as_uint(c)), "r"(__float_as_uint(d)),
               "r"(remote_mbar)
               : "memory");
}

// two packed pairs (c, c + 2) and (c + 1, c + 3) as the four floats of a row in column order
__device__ __forceinline__ float4 cols4(f32x2 v0, f32x2 v1) { return make_float4(lo2(v0), lo2(v1), hi2(v0), hi2(v1)); }

template <int FID, bool MASK>
__device__ __forceinline__ void fused_wrow_body(const LocalArgs& A, const int first, const int stride) {
  using L = WrLayout2;
  constexpr int NW = L::NW, CL = L::CL, BAND = L::BAND, BW = L::BW;
  extern __shared__ __align__(16) float smem[];
  const uint32_t mbU = smem_addr(smem + L::MB);
  const uint32_t mbQ = mbU + 8;
  const uint32_t mbL = mbU + 16;

  const Grid g = A.g;
  const int T = g.NR * g.NC;
  const int rank = (int)blockIdx.x;
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  const int tid = threadIdx.x;
  const int br0 = 2 * w;  // the warp's first row in the band
  const int W2 = g.W + g.NC;
  const float tau = A.tau;
  const int K = A.K;
  const bool tile_top_warp = rank == 0 && w == 0;      // holds the tile's first row
  const bool last_here = rank == CL - 1 && w == NW - 1;  // holds the tile's last row (bottom side below it)
  const bool push_down = w == NW - 1 && rank + 1 < CL;   // sends u of the band's last row
  const bool push_up = w == 0 && rank > 0;               // sends pbar1 of the band's first row
  const bool need_uh = push_up;
  const bool need_qh = push_down;
  constexpr uint32_t kHaloBytes = 4 * BW;
  uint32_t remote_u = 0, remote_q = 0, remote_mbU = 0, remote_mbQ = 0;
  if (push_down) {
    remote_u = map_rank(smem_addr(smem + L::UH + 4 * l), rank + 1);
    remote_mbU = map_rank(mbU, rank + 1);
  }
  if (push_up) {
    remote_q = map_rank(smem_addr(smem + L::QH + 4 * l), rank - 1);
    remote_mbQ = map_rank(mbQ, rank - 1);
  }
  if (tid == 0) {
    mbar_init(mbU, 1);
    mbar_init(mbQ, 1);
    mbar_init(mbL, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  for (int q = tid; q < 8 * min(K, L::kMaxSmemCoef); q += L::NT) smem[L::CO + q] = reinterpret_cast<const float*>(A.coef)[q];
  if (rank == 0 && w == 0) *reinterpret_cast<float4*>(smem + L::UH + 4 * l) = make_float4(0.f, 0.f, 0.f, 0.f);
  __syncthreads();
  if (need_uh && l == 0) mbar_arrive_expect_tx(mbU, kHaloBytes);
  if (need_qh && l == 0) mbar_arrive_expect_tx(mbQ, kHaloBytes);
  cluster_arrive<true>();  // barriers initialised and armed everywhere before any halo is sent
  cluster_wait();

  // bytes the prefetch of tile t brings into this CTA (the copies issued below)
  auto prefetch_bytes = [&](int a, int b) -> uint32_t {
    uint32_t n = BAND * (3 * 512 + 4 * L::P2S);
    if (rank == 0 && a > 0) n += 512;
    if (rank == CL - 1 && a + 1 < g.NR) n += 1024;
    if (rank < CL - 1) n += 512;
    if (b > 0) n += 64;
    if (b + 1 < g.NC) n += 64;
    return n;
  };
  // lane 0 of every warp copies the warp's two rows; warps 0 and NW - 1 the extras
  auto prefetch = [&](int t) {
    const int a = t / g.NC, b = t - a * g.NC;
    const int c0 = b * 128, gb = a * 128 + rank * BAND;
    if (tid == 0) mbar_arrive_expect_tx(mbL, prefetch_bytes(a, b));
    if (l == 0) {
      const int o = b & 3;  // p2 tile window starts 16-byte aligned, o floats before column c0 + b
#pragma unroll
      for (int r = 0; r < 2; ++r) {
        const int br = br0 + r, gi = gb + br;
        bulk_g2s(smem + L::SU + br * BW, A.u + (size_t)gi * g.W + c0, 512, mbL);
        bulk_g2s(smem + L::SU + BAND * BW + br * BW, A.f + (size_t)gi * g.W + c0, 512, mbL);
        bulk_g2s(smem + L::SU + 2 * BAND * BW + br * BW, A.P1 + (size_t)(gi + a) * g.W + c0, 512, mbL);
        bulk_g2s(smem + L::SP2 + br * L::P2S, A.P2 + (size_t)gi * W2 + c0 + b - o, 4 * L::P2S, mbL);
      }
      if (w == 0) {
        if (rank == 0 && a > 0) bulk_g2s(smem + L::XLT, A.lamh + (size_t)(a - 1) * g.W + c0, 512, mbL);
        if (b > 0) bulk_g2s(smem + L::XLL, A.lamv + (size_t)(b - 1) * g.H + gb, 64, mbL);
        if (b + 1 < g.NC) bulk_g2s(smem + L::XLR, A.lamv + (size_t)b * g.H + gb, 64, mbL);
      }
      if (w == NW - 1) {
        if (rank == CL - 1) {
          if (a + 1 < g.NR) {
            bulk_g2s(smem + L::XPB, A.P1 + (size_t)(a * 128 + 128 + a) * g.W + c0, 512, mbL);
            bulk_g2s(smem + L::XLB, A.lamh + (size_t)a * g.W + c0, 512, mbL);
          }
        } else {
          bulk_g2s(smem + L::XQH, A.P1 + (size_t)(gb + BAND + a) * g.W + c0, 512, mbL);
        }
      }
    }
  };

  bool timed_out = false;
  uint32_t phU = 0, phQ = 0;  // index of the next phase of mbU / mbQ this CTA waits for
  auto wait_u = [&]() {
    if (!mbar_wait(mbU, phU & 1)) timed_out = true;
    ++phU;
    if (l == 0) mbar_arrive_expect_tx(mbU, kHaloBytes);  // arm the next phase
  };
  auto wait_q = [&]() {
    if (!mbar_wait(mbQ, phQ & 1)) timed_out = true;
    ++phQ;
    if (l == 0) mbar_arrive_expect_tx(mbQ, kHaloBytes);
  };

  if (first < T) prefetch(first);
  uint32_t nsub = 0;  // subdomains this CTA has started (phase of mbL)

  for (int t = first; t < T; t += stride, ++nsub) {
    const int a = t / g.NC, b = t - a * g.NC;
    const int c0 = b * 128, gb = a * 128 + rank * BAND;
    const bool s_top = a > 0, s_bot = a + 1 < g.NR, s_lft = b > 0, s_rgt = b + 1 < g.NC;
    const int o = b & 3;
    const float lim_top = (tile_top_warp && !s_top) ? 0.f : 1.f;  // p1 of the tile's first row
    const float lim_left = (l == 0 && !s_lft) ? 0.f : 1.f;        // p2 of the tile's first column
    // pairs [row r][c]: columns (4l + c, 4l + c + 2) of band row br0 + r
    f32x2 U[2][2], P1[2][2], P2[2][2], H1[2][2], H2[2][2], Q1[2][2], Q2[2][2];
    f32x2 Bv[2] = {0ull, 0ull};                     // pbar1 of the row below the band (last CTA's last warp: bottom side)
    float pB[4] = {0.f, 0.f, 0.f, 0.f}, hB[4] = {0.f, 0.f, 0.f, 0.f};  // bottom side p, phat (last warp of last CTA)
    float pr[2] = {0.f, 0.f}, hr[2] = {0.f, 0.f}, qr[2] = {0.f, 0.f};  // right side p, phat, pbar (lane 31)
    uint32_t in_d = 0;  // bit 4r + col: pixel of row r, column 4l + col lies in the inpainting domain

    if (!mbar_wait(mbL, nsub & 1)) timed_out = true;  // staging of this subdomain landed
    __syncthreads();  // every warp has left the previous subdomain
    {
#pragma unroll
      for (int r = 0; r < 2; ++r) {
        const int br = br0 + r;
        const float4 uu = *reinterpret_cast<const float4*>(smem + L::SU + br * BW + 4 * l);
        float4 ff = *reinterpret_cast<const float4*>(smem + L::SU + BAND * BW + br * BW + 4 * l);
        const float4 p1 = *reinterpret_cast<const float4*>(smem + L::SU + 2 * BAND * BW + br * BW + 4 * l);
        const float* p2s = smem + L::SP2 + br * L::P2S + o + 4 * l;
        const float p2v[4] = {p2s[0], p2s[1], p2s[2], p2s[3]};
        if (FID == FID_SEG) {
          auto seg = [&](float v) { return (v - A.c1) * (v - A.c1) - (v - A.c2) * (v - A.c2); };
          ff = make_float4(seg(ff.x), seg(ff.y), seg(ff.z), seg(ff.w));
        }
        if (MASK) {
          const uint8_t* mrow = A.mask + (size_t)(gb + br) * g.W + c0 + 4 * l;
#pragma unroll
          for (int col = 0; col < 4; ++col)
            if (mrow[col]) in_d |= 1u << (4 * r + col);
        }
        float h1v[4] = {p1.x, p1.y, p1.z, p1.w};
        float h2v[4] = {p2v[0], p2v[1], p2v[2], p2v[3]};
        if (tile_top_warp && r == 0 && s_top) {
#pragma unroll
          for (int col = 0; col < 4; ++col) h1v[col] = phat_t(h1v[col], smem[L::XLT + 4 * l + col], tau);
        }
        if (l == 0 && s_lft) h2v[0] = phat_t(p2v[0], smem[L::XLL + br], tau);
        U[r][0] = pk2(uu.x, uu.z);
        U[r][1] = pk2(uu.y, uu.w);
        P1[r][0] = pk2(p1.x, p1.z);
        P1[r][1] = pk2(p1.y, p1.w);
        P2[r][0] = pk2(p2v[0], p2v[2]);
        P2[r][1] = pk2(p2v[1], p2v[3]);
        H1[r][0] = pk2(h1v[0], h1v[2]);
        H1[r][1] = pk2(h1v[1], h1v[3]);
        H2[r][0] = pk2(h2v[0], h2v[2]);
        H2[r][1] = pk2(h2v[1], h2v[3]);
        Q1[r][0] = P1[r][0];
        Q1[r][1] = P1[r][1];
        Q2[r][0] = P2[r][0];
        Q2[r][1] = P2[r][1];
        *reinterpret_cast<float4*>(smem + L::F + (w * 32 + l) * 8 + 4 * r) = make_float4(ff.x, ff.z, ff.y, ff.w);
        if (l == 31 && s_rgt) {
          pr[r] = smem[L::SP2 + br * L::P2S + o + 128];
          hr[r] = phat_s(pr[r], smem[L::XLR + br], tau);
          qr[r] = pr[r];
        }
      }
      // initial pbar1 of the warp's first row, read by the warp above in its u-step 0
      if (w > 0)
        *reinterpret_cast<float4*>(smem + L::QBUF + (w * 2 + 1) * BW + 4 * l) =
            make_float4(lo2(P1[0][0]), hi2(P1[0][0]), lo2(P1[0][1]), hi2(P1[0][1]));
      if (need_qh) {
        const float4 x = *reinterpret_cast<const float4*>(smem + L::XQH + 4 * l);
        *reinterpret_cast<float4*>(smem + L::QH + 4 * l) = make_float4(x.x, x.z, x.y, x.w);
      }
      if (last_here && s_bot) {
#pragma unroll
        for (int col = 0; col < 4; ++col) {
          pB[col] = smem[L::XPB + 4 * l + col];
          hB[col] = phat_s(pB[col], smem[L::XLB + 4 * l + col], tau);
        }
        Bv[0] = pk2(pB[0], pB[2]);
        Bv[1] = pk2(pB[1], pB[3]);
      }
    }
    __syncthreads();  // staging consumed by every warp; initial exchange values written
    if (t + stride < T) prefetch(t + stride);

    const float* myF = smem + L::F + (w * 32 + l) * 8;
    for (int k = 0; k < K; ++k) {
      Coef co;
      if (k < L::kMaxSmemCoef) {
        const float4 ca = *reinterpret_cast<const float4*>(smem + L::CO + 8 * k);
        const float4 cb = *reinterpret_cast<const float4*>(smem + L::CO + 8 * k + 4);
        co = Coef{ca.x, ca.y, ca.z, ca.w, cb.x, cb.y, cb.z, cb.w};
      } else {
        co = A.coef[k];
      }
      const f32x2 SIG = pk2(co.sig, co.sig), UA = pk2(co.ua, co.ua), UB = pk2(co.ub, co.ub);
      const f32x2 PA = pk2(co.pa, co.pa), PC = pk2(co.pc, co.pc), PB = pk2(co.pb, co.pb), TH = pk2(co.th, co.th);
      // ---------------- u-step: the warp's last row first
      if (w < NW - 1) {
        if (k > 0) bar_sync_n(8 + w, 64);  // Q(w + 1): pbar1 of the first row of the warp below
        const ulonglong2 qb =
            *reinterpret_cast<const ulonglong2*>(smem + L::QBUF + ((w + 1) * 2 + ((k + 1) & 1)) * BW + 4 * l);
        Bv[0] = qb.x;
        Bv[1] = qb.y;
      } else if (need_qh) {
        if (k > 0) wait_q();  // pbar1 halo of iteration k - 1
        const ulonglong2 qb = *reinterpret_cast<const ulonglong2*>(smem + L::QH + 4 * l);
        Bv[0] = qb.x;
        Bv[1] = qb.y;
      }
      const ulonglong2 fr0 = *reinterpret_cast<const ulonglong2*>(myF);
      const ulonglong2 fr1 = *reinterpret_cast<const ulonglong2*>(myF + 4);
#pragma unroll
      for (int rr = 0; rr < 2; ++rr) {
        const int r = 1 - rr;
        float nb = __shfl_down_sync(0xffffffffu, lo2(Q2[r][0]), 1);  // pbar2 of the edge left of column 4l + 4
        if (l == 31) nb = qr[r];                                    // the tile's right side
#pragma unroll
        for (int c = 0; c < 2; ++c) {
          const f32x2 below = r == 0 ? Q1[1][c] : Bv[c];
          const f32x2 right = c == 0 ? Q2[r][1] : pk2(hi2(Q2[r][0]), nb);
          const f32x2 d = sub2(add2(sub2(below, Q1[r][c]), right), Q2[r][c]);  // div_px
          const f32x2 fg = r == 0 ? (c == 0 ? fr0.x : fr0.y) : (c == 0 ? fr1.x : fr1.y);
          const f32x2 ub = fma2(SIG, d, U[r][c]);
          const bool dl = MASK && ((in_d >> (4 * r + c)) & 1u), dh = MASK && ((in_d >> (4 * r + c + 2)) & 1u);
          f32x2 un;
          if (FID == FID_L2) {
            un = fma2(UB, fg, mul2(UA, ub));
            if (MASK) un = pk2(dl ? lo2(ub) : lo2(un), dh ? hi2(ub) : hi2(un));
          } else {
            un = pk2(prox_ubar<FID>(lo2(ub), lo2(fg), dl, co), prox_ubar<FID>(hi2(ub), hi2(fg), dh, co));
          }
          U[r][c] = un;
        }
        if (r == 1) {
          if (w < NW - 1) {
            *reinterpret_cast<ulonglong2*>(smem + L::UBUF + (w * 2 + (k & 1)) * BW + 4 * l) =
                make_ulonglong2(U[1][0], U[1][1]);
            bar_arrive_n(1 + w, 64);  // U(w)
          } else if (push_down) {
            st_async_v4(remote_u, lo2(U[1][0]), hi2(U[1][0]), lo2(U[1][1]), hi2(U[1][1]), remote_mbU);
          }
        }
      }
      // ---------------- p-step: the warp's first row first
      f32x2 Av[2];
      if (w > 0) {
        bar_sync_n(w, 64);  // U(w - 1): u of the last row of the warp above
        const ulonglong2 ua =
            *reinterpret_cast<const ulonglong2*>(smem + L::UBUF + ((w - 1) * 2 + (k & 1)) * BW + 4 * l);
        Av[0] = ua.x;
        Av[1] = ua.y;
      } else {
        if (need_uh) wait_u();  // u halo of iteration k
        const ulonglong2 ua = *reinterpret_cast<const ulonglong2*>(smem + L::UH + 4 * l);
        Av[0] = ua.x;
        Av[1] = ua.y;
      }
#pragma unroll
      for (int r = 0; r < 2; ++r) {
        float nu = __shfl_up_sync(0xffffffffu, hi2(U[r][1]), 1);  // u of column 4l - 1
        if (l == 0) nu = 0.f;                                     // left of the tile
#pragma unroll
        for (int c = 0; c < 2; ++c) {
          const f32x2 above = r == 0 ? Av[c] : U[0][c];
          const f32x2 leftu = c == 1 ? U[r][0] : pk2(nu, lo2(U[r][1]));
          {
            const f32x2 tt = fma2(PC, sub2(U[r][c], above), fma2(PA, P1[r][c], mul2(PB, H1[r][c])));  // p_target
            const float lt = r == 0 ? lim_top : 1.f;
            const f32x2 pn = pk2(fminf(fmaxf(lo2(tt), -lt), lt), fminf(fmaxf(hi2(tt), -lt), lt));
            Q1[r][c] = fma2(TH, sub2(pn, P1[r][c]), pn);
            P1[r][c] = pn;
          }
          {
            const f32x2 tt = fma2(PC, sub2(U[r][c], leftu), fma2(PA, P2[r][c], mul2(PB, H2[r][c])));
            const float ll = c == 0 ? lim_left : 1.f;
            const f32x2 pn = pk2(fminf(fmaxf(lo2(tt), -ll), ll), fminf(fmaxf(hi2(tt), -1.f), 1.f));
            Q2[r][c] = fma2(TH, sub2(pn, P2[r][c]), pn);
            P2[r][c] = pn;
          }
        }
        if (r == 0) {
          if (w > 0) {
            if (k < K - 1) {
              *reinterpret_cast<ulonglong2*>(smem + L::QBUF + (w * 2 + (k & 1)) * BW + 4 * l) =
                  make_ulonglong2(Q1[0][0], Q1[0][1]);
              bar_arrive_n(8 + w - 1, 64);  // Q(w)
            }
          } else if (push_up) {
            st_async_v4(remote_q, lo2(Q1[0][0]), hi2(Q1[0][0]), lo2(Q1[0][1]), hi2(Q1[0][1]), remote_mbQ);
          }
        }
      }
      if (l == 31 && s_rgt) {
#pragma unroll
        for (int r = 0; r < 2; ++r) p_update(pr[r], qr[r], -hi2(U[r][1]), hr[r], co);
      }
      if (last_here && s_bot) {
        float qB[4];
        const float ul[4] = {lo2(U[1][0]), lo2(U[1][1]), hi2(U[1][0]), hi2(U[1][1])};
#pragma unroll
        for (int col = 0; col < 4; ++col) p_update(pB[col], qB[col], -ul[col], hB[col], co);
        Bv[0] = pk2(qB[0], qB[2]);
        Bv[1] = pk2(qB[1], qB[3]);
      }
    }
    if (need_qh) wait_q();  // drain the last pbar1 halo (not read)

    // ---- write back: u and p1 through shared memory and bulk copies, p2 and the sides directly
    if (l == 0) bulk_wait_read();  // the previous subdomain's outgoing rows have been read
    __syncwarp();
#pragma unroll
    for (int r = 0; r < 2; ++r) {
      const int br = br0 + r;
      *reinterpret_cast<float4*>(smem + L::SOU + br * BW + 4 * l) = cols4(U[r][0], U[r][1]);
      *reinterpret_cast<float4*>(smem + L::SOP + br * BW + 4 * l) = cols4(P1[r][0], P1[r][1]);
      float* p2row = A.P2 + (size_t)(gb + br) * W2 + c0 + b + 4 * l;
      p2row[0] = lo2(P2[r][0]);
      p2row[1] = lo2(P2[r][1]);
      p2row[2] = hi2(P2[r][0]);
      p2row[3] = hi2(P2[r][1]);
      if (l == 0 && s_lft) A.out.SL[(size_t)(b - 1) * g.H + gb + br] = lo2(P2[r][0]);
      if (l == 31 && s_rgt) {
        A.P2[(size_t)(gb + br) * W2 + c0 + 128 + b] = pr[r];
        A.out.SR[(size_t)b * g.H + gb + br] = pr[r];
      }
    }
    if (tile_top_warp && s_top)
      *reinterpret_cast<float4*>(A.out.ST + (size_t)(a - 1) * g.W + c0 + 4 * l) = cols4(P1[0][0], P1[0][1]);
    if (last_here && s_bot) {
      const float4 v = make_float4(pB[0], pB[1], pB[2], pB[3]);
      *reinterpret_cast<float4*>(A.P1 + (size_t)(a * 128 + 128 + a) * g.W + c0 + 4 * l) = v;
      *reinterpret_cast<float4*>(A.out.SB + (size_t)a * g.W + c0 + 4 * l) = v;
    }
    fence_proxy_async();  // the rows written above become visible to the bulk copies
    __syncwarp();
    if (l == 0) {
#pragma unroll
      for (int r = 0; r < 2; ++r) {
        const int br = br0 + r, gi = gb + br;
        bulk_s2g(A.u + (size_t)gi * g.W + c0, smem + L::SOU + br * BW, 512);
        bulk_s2g(A.P1 + (size_t)(gi + a) * g.W + c0, smem + L::SOP + br * BW, 512);
      }
      bulk_commit();
    }
  }
  if (l == 0) bulk_wait_all();  // outgoing rows written before the CTA's shared memory is released
  cluster_arrive<true>();       // no CTA leaves while a neighbour may still write into it
  cluster_wait();
  if (timed_out) atomicOr(A.err, 1);
}

template <int FID, bool MASK>
__global__ void __launch_bounds__(WrLayout2::NT, 2) k_fused_wrow(const LocalArgs A) {
  fused_wrow_body<FID, MASK>(A, blockIdx.y, gridDim.y);
}

template <int FID, bool MASK>
int& wrow_clusters(int dev) {
  static int n[64] = {0};
  return n[dev & 63];
}

cudaLaunchConfig_t wrow_config(int clusters, cudaLaunchAttribute* attr) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(WrLayout2::CL, clusters, 1);
  cfg.blockDim = dim3(WrLayout2::NT, 1, 1);
  cfg.dynamicSmemBytes = WrLayout2::BYTES;
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = WrLayout2::CL;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cfg;
}

template <int FID, bool MASK>
cudaError_t prepare_wrow_one() {
  auto kern = k_fused_wrow<FID, MASK>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)WrLayout2::BYTES);
  if (e != cudaSuccess) return e;
  cudaLaunchAttribute attr[1];
  cudaLaunchConfig_t cfg = wrow_config(1024, attr);
  int n = 0;
  if (cudaOccupancyMaxActiveClusters(&n, kern, &cfg) != cudaSuccess) {
    cudaGetLastError();
    n = 0;
  }
  int dev = 0;
  cudaGetDevice(&dev);
  wrow_clusters<FID, MASK>(dev) = n;
  return cudaSuccess;
}

template <int FID, bool MASK>
cudaError_t launch_wrow_one(const LocalArgs& a, cudaStream_t st) {
  int dev = 0;
  cudaGetDevice(&dev);
  const int tiles = a.g.NR * a.g.NC;
  int nc = wrow_clusters<FID, MASK>(dev);
  if (nc <= 0 || nc > tiles) nc = tiles;
  cudaLaunchAttribute attr[1];
  cudaLaunchConfig_t cfg = wrow_config(nc, attr);
  cfg.stream = st;
  return cudaLaunchKernelEx(&cfg, k_fused_wrow<FID, MASK>, a);
}

}  // namespace

bool fused_wrow_supported(const LocalArgs& a) {
  auto al16 = [](const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15) == 0; };
  return a.g.H == 128 * a.g.NR && a.g.W == 128 * a.g.NC && (a.g.W + a.g.NC) % 4 == 0 && al16(a.u) && al16(a.f) &&
         al16(a.P1) && al16(a.P2) && al16(a.lamh) && al16(a.lamv) && al16(a.out.ST) && al16(a.out.SB) &&
         (a.mask == nullptr || (reinterpret_cast<uintptr_t>(a.mask) & 3) == 0);
}

cudaError_t fused_wrow_prepare() {
  cudaError_t e;
  if ((e = prepare_wrow_one<FID_L2, false>()) != cudaSuccess) return e;
  if ((e = prepare_wrow_one<FID_L2, true>()) != cudaSuccess) return e;
  if ((e = prepare_wrow_one<FID_L1, false>()) != cudaSuccess) return e;
  if ((e = prepare_wrow_one<FID_L1, true>()) != cudaSuccess) return e;
  return prepare_wrow_one<FID_SEG, false>();
}

cudaError_t launch_fused_wrow(const LocalArgs& a, int fid, cudaStream_t st) {
  const bool m = a.mask != nullptr;
  switch (fid) {
    case FID_L2: return m ? launch_wrow_one<FID_L2, true>(a, st) : launch_wrow_one<FID_L2, false>(a, st);
    case FID_L1: return m ? launch_wrow_one<FID_L1, true>(a, st) : launch_wrow_one<FID_L1, false>(a, st);
    default: return launch_wrow_one<FID_SEG, false>(a, st);
  }
}

}  // namespace ddtv
