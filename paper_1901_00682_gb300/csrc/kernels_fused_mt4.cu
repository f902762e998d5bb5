// Persistent fused local solver on 4 x 4 micro-tiles, one warp per thread row
// (128 x 128 subdomains).
//
// The 2 x 4 micro-tile kernel (kernels_fused_mt.cu) holds 8 pixels per thread in
// 256-thread CTAs, two per SM.  Here a thread holds a micro-tile of four columns by
// four rows (16 pixels), so per pixel half as many edge values cross between threads,
// and a warp holds four full rows of the CTA's band: the exchange between horizontal
// neighbours never leaves the warp.  A CTA is four warps (128 threads) covering a band
// of 16 rows; with up to 170 registers per thread three CTAs fit on an SM, which then
// interleaves three subdomain bands instead of two.  The tile's right side (the p2 dofs
// of column 128) is updated by lanes 0..15 of warp 1, one band row each, in registers;
// the bottom side by warp 2 of the last CTA.
//
// Per inner iteration a lane exchanges, with one 16-byte shared-memory access each, the
// u of its right column (for the lane to its right), the pbar2 of its left edge (for
// the lane to its left), and its warp's last-row u and first-row pbar1 with the warps
// above and below; two CTA barriers order them.  Rows crossing CTAs travel with
// st.async and mbarrier complete_tx (bounded waits, the same phase protocol as
// kernels_fused_mt.cu), and the next subdomain is prefetched with 16-byte cp.async copies
// (p2 as a window starting on a 16-byte boundary: W + N_c must be a multiple of 4).
// Rows are packed in pairs (r, r + 2) for the `*.f32x2` arithmetic; every value is
// computed with the operations of the scalar iteration in the same order, so the
// results are bit-identical to the other mappings.
//
// TMA: the same kernel moving the state with the tensor memory accelerator.  One thread
// loads the next subdomain's u, f, p1 bands and p2 window as four 2-D tensor copies
// (cp.async.bulk.tensor, completion counted on an mbarrier), and stores the previous
// subdomain's u and p1 bands from an out-buffer in shared memory as two tensor copies
// (bulk group, issued after the barrier that follows the out-buffer writes; the buffer
// is rewritten only after a wait for the copies to have read it); p2 and the sides go
// out with ordinary stores.
//
// Batch: k_fused_mt4_batch runs the cp.async form of the body over the work list of a
// batch of images (BatchTiles), every subdomain with its image's descriptor (kept in
// shared memory while the image does not change), fidelity and coefficients.
//
// ADAPT (tensor-copy kernel only): adaptive inner stopping (Section 5, eq. stop_inner1).
// Every thread sums (p^{k+1} - p^k)^2 and (p^{k+1})^2 over its dofs in the p-step of
// iteration k (packed float32 pairs) and leaves them in the P1 out-buffer, idle during
// the inner loop.  At the start of iteration k + 1 one warp adds the CTA's 128 pairs
// (float32, fixed order) and sends the CTA's pair with st.async to slot `rank` of every
// CTA of the cluster, counted on one of two mbarriers (by the parity of the phase, so
// that a phase is always consumed everywhere before its barrier is armed again).  Before
// the barrier between the u-step and the p-step of iteration k + 1, one warp per CTA
// waits for the CL pairs and adds them in a fixed tree: every CTA takes the same
// decision without a cluster barrier.  On "stop" the u-step of iteration k + 1 is undone
// (each iteration first copies u into the u out-buffer, which then already holds the
// result), its u halo is drained and the p-step is skipped: the solve keeps k + 1 inner
// iterations, as the rule prescribes.
#include <cuda.h>

#include "fused_common.cuh"
#include "internal.cuh"

namespace ddtv {

namespace {

struct Mt4Layout {
  static constexpr int CL = 8, NW = 4, BAND = 4 * NW, BW = 128, NT = 32 * NW;
  static constexpr int P2S = 132;                    // staged p2 row: 132 floats from a 16-byte boundary
  static constexpr int SLOT = 4 * 33;                // one warp's UR / QL slots
  // (NW + 1) x 128, column order: row 0 = u of the row above the band (halo; zero in
  // the first CTA), row w + 1 = u of warp w's last row
  static constexpr int UB = 0;
  // (NW + 1) x 128, column order: row w = pbar1 of warp w's first row, row NW = pbar1
  // of the row below the band (halo, or the tile's bottom side)
  static constexpr int Q1 = UB + (NW + 1) * BW;
  // NW x 33 x 4, pair order: slot 0 = zero (left of the tile), slot l + 1 = u of lane
  // l's right column
  static constexpr int UR = Q1 + (NW + 1) * BW;
  static constexpr int QL = UR + NW * SLOT;          // NW x 33 x 4: slot l = pbar2 of lane l's left edge
  static constexpr int F = QL + NW * SLOT;           // NW x 4 (column) x 32 (lane) x 4: f (or g), pair order
  // kMaxSmemCoef x 16: the 8 coefficients of each inner iteration, each stored twice
  // (sig sig ua ua ub ub s s pa pa pc pc pb pb th th) so that one 16-byte load gives two
  // packed pairs
  static constexpr int CO = F + NW * 4 * 32 * 4;
  static constexpr int kMaxSmemCoef = 64;
  static constexpr int SU = CO + 16 * kMaxSmemCoef;  // staging of the next subdomain: u, f, p1 (BAND x 128 each)
  static constexpr int SP2 = SU + 3 * BAND * BW;     // p2 window (BAND x P2S)
  static constexpr int XLT = SP2 + BAND * P2S;       // lamh above the tile (128)
  static constexpr int XPB = XLT + BW;               // p1 of the tile's bottom side (128)
  static constexpr int XLB = XPB + BW;               // lamh below the tile (128)
  static constexpr int XQH = XLB + BW;               // p1 of the first row below the band (128); in the
                                                     // last CTA, which has no band below: u of the tile's last row
  static constexpr int XLL = XQH + BW;               // lamv left of the band rows (BAND)
  static constexpr int XLR = XLL + BAND;             // lamv right of the band rows (BAND)
  static constexpr int PBS = XLR + BAND;             // bottom side p of the tile (128; last CTA)
  static constexpr int HBS = PBS + BW;               // bottom side phat (128)
  static constexpr int MB = HBS + BW;                // two mbarriers
  static constexpr size_t BYTES = sizeof(float) * MB + 16;
  // tensor-copy variant: out-buffers of u and p1 (128-byte aligned), three mbarriers
  static constexpr int OU = (HBS + BW + 31) & ~31;
  static constexpr int OP1 = OU + BAND * BW;
  // adaptive inner stop: during the inner loop OP1 holds every thread's residual sums (4
  // floats per thread); two buffers (one per parity of the reduction phase) of CL
  // slots, one (sum (dp)^2, sum p^2) pair per CTA of the cluster; the CTA's decision
  static constexpr int PS = OP1;
  static constexpr int RED = OP1 + BAND * BW;
  static constexpr uint32_t kRedBytes = 8 * CL;  // one phase: every CTA's pair
  static constexpr int STOP = RED + 2 * 2 * CL;
  static constexpr int MBT = STOP + 2;           // five mbarriers
#ifndef MT4_REDUCE_WARP
#define MT4_REDUCE_WARP 3
#endif
#ifndef MT4_DECIDE_WARP
#define MT4_DECIDE_WARP 1
#endif
  static constexpr int kReduceWarp = MT4_REDUCE_WARP;  // adds the CTA's residual sums and sends them
  static constexpr int kDecideWarp = MT4_DECIDE_WARP;  // takes the stop decision
  static constexpr size_t BYTES_TMA = sizeof(float) * MBT + 48;
  static constexpr uint32_t kTmaBytes = 4 * (3 * BAND * BW + BAND * P2S);  // one subdomain's four tensor loads
  static_assert(Q1 % 4 == 0 && UR % 4 == 0 && QL % 4 == 0 && F % 4 == 0 && CO % 4 == 0 && SU % 4 == 0 &&
                    SP2 % 4 == 0 && XLT % 4 == 0 && XLL % 4 == 0 && XLR % 4 == 0 && PBS % 4 == 0 &&
                    HBS % 4 == 0 && MB % 2 == 0,
                "16-byte alignment of the vector and cp.async buffers");
  static_assert(CL * BAND == 128, "a cluster of CTAs covers the 128 rows of a tile");
  static_assert(SU % 32 == 0 && SP2 % 32 == 0 && (BAND * BW) % 32 == 0 && OU % 32 == 0 && OP1 % 32 == 0,
                "tensor copies need 128-byte aligned shared memory");
  static_assert(RED % 2 == 0 && MBT % 2 == 0, "8-byte alignment of the reduction slots and mbarriers");
  static_assert(4 * NT <= BAND * BW, "the residual sums of every thread fit the P1 out-buffer");
};

// tensor maps of the state arrays: u, f, p1 with 128 x 16 boxes, p2 with 132 x 16 boxes
struct Mt4Maps {
  CUtensorMap u, f, p1, p2;
};

__device__ __forceinline__ void tma_load_2d(float* dst, const CUtensorMap* map, int x, int y, uint32_t mbar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::
          "r"(smem_addr(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(mbar)
      : "memory");
}
__device__ __forceinline__ void tma_store_2d(const CUtensorMap* map, const float* src, int x, int y) {
  asm volatile("cp.async.bulk.tensor.2d.global.shared::cta.tile.bulk_group [%0, {%1, %2}], [%3];" ::"l"(
                   reinterpret_cast<uint64_t>(map)),
               "r"(x), "r"(y), "r"(smem_addr(src))
               : "memory");
}
__device__ __forceinline__ void tma_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
__device__ __forceinline__ void tma_wait_read() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }
__device__ __forceinline__ void tma_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }
__device__ __forceinline__ void tma_fence_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ float lane4(f32x2 v, int h) { return h ? hi2(v) : lo2(v); }

// The subdomains of one image (tile t = a N_c + b), its fidelity fixed at compile time.
// The batch kernel runs the same body over BatchTiles (fused_common.cuh): every
// subdomain with its image's geometry, parameters, strips and fidelity.
template <int FID>
struct Mt4One {
  const LocalArgs& A;
  static constexpr bool kBatch = false;
  __device__ int count() const { return A.g.NR * A.g.NC; }
  __device__ int inner() const { return A.K; }
  __device__ int image(int) const { return 0; }
  __device__ const LocalArgs& args(int) const { return A; }
  __device__ int local(int t) const { return t; }
  __device__ Strips out(int) const { return A.out; }
  __device__ int* err() const { return A.err; }
  template <class Body>
  __device__ void dispatch(int, Body&& body) const {
    body(FidC<FID>{});
  }
};

// A batch image's descriptor as the batch kernel keeps it in shared memory: its
// LocalArgs, the strips it writes this launch, its first tile in the work list, its
// fidelity and its index.
struct Mt4BatchDesc {
  LocalArgs A;
  Strips out;
  int base, fid, img, pad;
};
static_assert(sizeof(LocalArgs) % 4 == 0 && sizeof(Strips) % 4 == 0 && sizeof(Mt4BatchDesc) % 16 == 0,
              "descriptors copied word by word");

// every thread of the CTA copies words of image img's descriptor into d (a barrier must
// follow before d is read)
__device__ __forceinline__ void load_batch_desc(Mt4BatchDesc* d, const BatchArgs& B, int img, int tid, int nt) {
  constexpr int kA = sizeof(LocalArgs) / 4, kS = sizeof(Strips) / 4, kN = sizeof(Mt4BatchDesc) / 4;
  const uint32_t* a = reinterpret_cast<const uint32_t*>(B.args + img);
  const uint32_t* st = reinterpret_cast<const uint32_t*>(B.strips + 2 * img + B.write_set);
  uint32_t* dst = reinterpret_cast<uint32_t*>(d);
  for (int q = tid; q < kN; q += nt) {
    uint32_t v = 0;
    if (q < kA) v = a[q];
    else if (q < kA + kS) v = st[q - kA];
    else if (q == kA + kS) v = (uint32_t)B.tile_base[img];
    else if (q == kA + kS + 1) v = (uint32_t)B.fid[img];
    else if (q == kA + kS + 2) v = (uint32_t)img;
    dst[q] = v;
  }
}

// the coefficient sets of an image into shared memory, each coefficient twice
__device__ __forceinline__ void load_coef_dup(float* sCo, const Coef* coef, int K, int tid, int nt) {
  for (int q = tid; q < 16 * K; q += nt)  // K <= kMaxSmemCoef
    sCo[q] = reinterpret_cast<const float*>(coef)[(q >> 4) * 8 + ((q & 15) >> 1)];
}

template <bool MASK, bool TMA, bool ADAPT, class Src>
__device__ __forceinline__ void fused_mt4_body(const Src& S, const Mt4Maps* M, const int first, const int stride) {
  using L = Mt4Layout;
  constexpr int NW = L::NW, CL = L::CL, BAND = L::BAND, NT = L::NT, BW = L::BW;
  extern __shared__ __align__(128) float smem[];
  float* sUB = smem + L::UB;
  float* sQ1 = smem + L::Q1;
  float* sCo = smem + L::CO;
  const uint32_t mbU = smem_addr(smem + (TMA ? L::MBT : L::MB));
  const uint32_t mbQ = mbU + 8;
  const uint32_t mbL = mbU + 16;  // tensor loads of the staged subdomain (TMA)
  const uint32_t mbR = mbU + 24;  // reduction phases of the adaptive stop, two mbarriers (parity)
  static_assert(!ADAPT || TMA, "the adaptive stop keeps the rolled-back u in the tensor-copy out-buffer");
  static_assert(!(Src::kBatch && (TMA || ADAPT || MASK)), "the batch runs the cp.async kernel, fixed counts, no mask");

  const int T = S.count();
  const int rank = (int)blockIdx.x;
  const int tid = threadIdx.x, w = tid >> 5, l = tid & 31;
  const int j0 = 4 * l;              // the lane's first column in the tile
  const int lr0 = 4 * w;             // the warp's first row in the band
  const int i0 = rank * BAND + lr0;  // ... in the tile
  const int K = S.inner();
  const bool last_row_here = rank == CL - 1 && w == NW - 1;
  // the tile's bottom side is updated by warp 2 of the last CTA (the last warp, which
  // holds the last row, already waits for halos and pushes rows); warp 1 updates the
  // right side
  const bool bottom_warp = rank == CL - 1 && w == 2;
  const bool push_down = w == NW - 1 && rank + 1 < CL;  // sends u of the band's last row
  const bool push_up = w == 0 && rank > 0;              // sends pbar1 of the band's first row
  const bool need_uh = push_up;
  const bool need_qh = push_down;
  constexpr uint32_t kHaloBytes = 4 * BW;
  float* const myUR = smem + L::UR + w * L::SLOT + 4 * (l + 1);
  float* const myQL = smem + L::QL + w * L::SLOT + 4 * l;
  float* const myF = smem + L::F + (w * 4 * 32 + l) * 4;  // column c at + c * 128
  uint32_t remote_u = 0, remote_q1 = 0, remote_mbU = 0, remote_mbQ = 0;
  if (push_down) {
    remote_u = map_rank(smem_addr(sUB + j0), rank + 1);
    remote_mbU = map_rank(mbU, rank + 1);
  }
  if (push_up) {
    remote_q1 = map_rank(smem_addr(sQ1 + NW * BW + j0), rank - 1);
    remote_mbQ = map_rank(mbQ, rank - 1);
  }
  if (tid == 0) {
    mbar_init(mbU, 1);
    mbar_init(mbQ, 1);
    if (TMA) mbar_init(mbL, 1);
    if (ADAPT) {
      mbar_init(mbR, 1);
      mbar_init(mbR + 8, 1);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (!Src::kBatch) load_coef_dup(sCo, S.args(0).coef, K, tid, NT);
  int cur_img = Src::kBatch ? -1 : 0;  // image whose coefficients are in sCo
  // batch: the descriptors of the current and of the next subdomain's image, in the P1
  // out-buffer region (unused by the cp.async kernel); a subdomain of the image already
  // held reuses its slot, so the work list is read from global memory once per subdomain
  // (its image index, loaded a subdomain ahead) and a descriptor once per image change
  Mt4BatchDesc* const dsc = reinterpret_cast<Mt4BatchDesc*>(smem + L::OP1);
  int cur = 0;  // slot of the current subdomain's descriptor
  if constexpr (Src::kBatch) {
    if (first < T) load_batch_desc(&dsc[0], S.B, S.B.tile_img[first], tid, NT);
  }
  if (rank == 0 && w == 0) *reinterpret_cast<float4*>(sUB + j0) = make_float4(0.f, 0.f, 0.f, 0.f);  // u above the tile
  if (l < 4) smem[L::UR + w * L::SLOT + l] = 0.f;  // u left of the tile
  __syncthreads();
  if (need_uh && l == 0) mbar_arrive_expect_tx(mbU, kHaloBytes);
  if (need_qh && l == 0) mbar_arrive_expect_tx(mbQ, kHaloBytes);
  if (ADAPT && tid == 32 * L::kDecideWarp) {  // lane 0 of the deciding warp arms both reduction barriers
    mbar_arrive_expect_tx(mbR, L::kRedBytes);
    mbar_arrive_expect_tx(mbR + 8, L::kRedBytes);
  }
  cluster_arrive<true>();  // barriers initialised and armed everywhere before any halo is sent
  cluster_wait();

  auto prefetch = [&](int t, const LocalArgs& A, const int lt) {
    const Grid g = A.g;
    const int W2 = g.W + g.NC;
    const int a = lt / g.NC, b = lt - a * g.NC;
    const int c0 = b * 128;
    const int gb = a * 128 + rank * BAND;  // image row of the band's first row
    if (TMA) {
      if (tid == 0) {
        mbar_arrive_expect_tx(mbL, L::kTmaBytes);
        tma_load_2d(smem + L::SU, &M->u, c0, gb, mbL);
        tma_load_2d(smem + L::SU + BAND * BW, &M->f, c0, gb, mbL);
        tma_load_2d(smem + L::SU + 2 * BAND * BW, &M->p1, c0, gb + a, mbL);
        tma_load_2d(smem + L::SP2, &M->p2, c0 + b - (b & 3), gb, mbL);
      }
    } else {
#pragma unroll
      for (int m = 0; m < 12; ++m) {  // u, f, p1: 3 x BAND rows x 32 chunks of 16 bytes
        const int fld = m >> 2;
        const int q = tid + NT * (m & 3);
        const int row = q >> 5, ch = q & 31;
        const float* base = fld == 0 ? A.u : (fld == 1 ? A.f : A.P1);
        const int grow = gb + row + (fld == 2 ? a : 0);
        cp_async16(smem + L::SU + fld * BAND * BW + row * BW + 4 * ch, base + (size_t)grow * g.W + c0 + 4 * ch);
      }
      if (!Src::kBatch || (W2 & 3) == 0) {
#pragma unroll
        for (int m = 0; m < 5; ++m) {  // p2 window: BAND rows x 33 chunks
          const int q = tid + NT * m;
          if (q < BAND * 33) {
            const int row = q / 33, ch = q - row * 33;
            cp_async16(smem + L::SP2 + row * L::P2S + 4 * ch,
                       A.P2 + (size_t)(gb + row) * W2 + c0 + b - (b & 3) + 4 * ch);
          }
        }
      } else {  // rows not 16-byte aligned (a batch image with W + N_c not a multiple of 4):
                // the tile's 129 p2 columns one by one, at the same place in the window
        const int o = b & 3;
        for (int q = tid; q < BAND * 129; q += NT) {
          const int row = q / 129, col = q - row * 129;
          cp_async4(smem + L::SP2 + row * L::P2S + o + col, A.P2 + (size_t)(gb + row) * W2 + c0 + b + col);
        }
      }
    }
    if (tid < 32) {
      if (rank == 0 && (a > 0 || g.cut_top)) cp_async16(smem + L::XLT + 4 * tid, A.lamh + (ptrdiff_t)(a - 1) * g.W + c0 + 4 * tid);
      if (tid < 4 && b > 0) cp_async16(smem + L::XLL + 4 * tid, A.lamv + (size_t)(b - 1) * g.H + gb + 4 * tid);
    } else if (tid < 64) {
      const int q = tid - 32;
      if (rank == CL - 1 && (a + 1 < g.NR || g.cut_bot))
        cp_async16(smem + L::XPB + 4 * q, A.P1 + (size_t)(a * 128 + 128 + a) * g.W + c0 + 4 * q);
      if (q < 4 && b + 1 < g.NC) cp_async16(smem + L::XLR + 4 * q, A.lamv + (size_t)b * g.H + gb + 4 * q);
    } else if (tid < 96) {
      const int q = tid - 64;
      if (rank == CL - 1 && (a + 1 < g.NR || g.cut_bot)) cp_async16(smem + L::XLB + 4 * q, A.lamh + (size_t)a * g.W + c0 + 4 * q);
    } else {
      const int q = tid - 96;
      if (rank < CL - 1) cp_async16(smem + L::XQH + 4 * q, A.P1 + (size_t)(gb + BAND + a) * g.W + c0 + 4 * q);
    }
    cp_async_commit();
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

  if (first < T) {
    if constexpr (Src::kBatch)
      prefetch(first, dsc[0].A, first - dsc[0].base);
    else
      prefetch(first, S.args(first), S.local(first));
  }
  uint32_t nsub = 0;             // subdomains started (phase of mbL)
  int pa = -1, pc0 = 0, pgb = 0;  // previous subdomain, whose u and p1 wait in the out-buffer (TMA)
  uint32_t gred = 0;              // adaptive stop: reduction phases sent (and consumed) so far

  for (int t = first; t < T; t += stride, ++nsub) {
    const LocalArgs& A = Src::kBatch ? dsc[cur].A : S.args(t);
    const Grid g = A.g;
    const int W2 = g.W + g.NC;
    const float tau = A.tau;
    const Strips out = Src::kBatch ? dsc[cur].out : S.out(t);
    const int lt = Src::kBatch ? t - dsc[cur].base : S.local(t);
    // batch: the next subdomain's image, loaded while this one's staging lands
    const int img_next = (Src::kBatch && t + stride < T) ? S.image(t + stride) : 0;
    const int a = lt / g.NC, b = lt - a * g.NC;
    const int c0 = b * 128;
    const int gb = a * 128 + rank * BAND;
    const int o = b & 3;
    const bool s_top = a > 0 || g.cut_top, s_bot = a + 1 < g.NR || g.cut_bot, s_lft = b > 0, s_rgt = b + 1 < g.NC;
    const float lim_left = (l == 0 && !s_lft) ? 0.f : 1.f;
    const float lim_top = (i0 == 0 && !s_top) ? 0.f : 1.f;
    // The tile's right side (the p2 dofs of column 128, one per band row) is updated by
    // lanes 0..15 of warp 1, lane i for band row i, which keeps its p and proximal
    // centre in registers; it reads the u of column 127 from the UR slot after lane 31's
    // and writes pbar into the QL slot after lane 31's, where lane 31 reads its right
    // neighbour's left edge.  Slot entries are in pair order: rows (0, 2, 1, 3).
    const bool right_rows = s_rgt && w == 1 && l < BAND;
    const int r_slot = (l >> 2) * L::SLOT + 4 * 32 + 2 * (l & 1) + ((l >> 1) & 1);
    float pr_s = 0.f, hr_s = 0.f;
    auto body = [&](auto fidc) {
    constexpr int FID = decltype(fidc)::value;
    // pairs [column c][e]: rows (e, e + 2) of column j0 + c
    f32x2 U[4][2], P1[4][2], P2[4][2], H1[4][2], H2[4][2], Q1[4][2], Q2[4][2];
    uint32_t in_d = 0;  // bit 4c + r: pixel (row r, column j0 + c) lies in the inpainting domain
    int k_run = K;  // adaptive stop: inner iterations kept (< K: u of the last u-step undone)

    cp_async_wait_all();
    if (TMA && !mbar_wait(mbL, nsub & 1)) timed_out = true;
    __syncthreads();  // staging landed; the previous subdomain's shared arrays are free
    if (Src::kBatch && dsc[cur].img != cur_img) {  // visible after the barrier that follows the unpack
      load_coef_dup(sCo, A.coef, K, tid, NT);
      cur_img = dsc[cur].img;
    }
    if (TMA && tid == 0 && pa >= 0) {  // the previous subdomain's u and p1 bands
      tma_store_2d(&M->u, smem + L::OU, pc0, pgb);
      tma_store_2d(&M->p1, smem + L::OP1, pc0, pgb + pa);
      tma_commit();
    }
    {
      f32x2 FV[4][2];
#pragma unroll
      for (int e = 0; e < 2; ++e) {  // rows e and e + 2 form the pairs of index e
        float u[2][4], fv[2][4], p1[2][4], p2[2][4];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int r = e + 2 * h, br = lr0 + r;
          const float4 uu = *reinterpret_cast<const float4*>(smem + L::SU + br * BW + j0);
          const float4 ff = *reinterpret_cast<const float4*>(smem + L::SU + BAND * BW + br * BW + j0);
          const float4 pp = *reinterpret_cast<const float4*>(smem + L::SU + 2 * BAND * BW + br * BW + j0);
          const float* p2s = smem + L::SP2 + br * L::P2S + o + j0;
          u[h][0] = uu.x;
          u[h][1] = uu.y;
          u[h][2] = uu.z;
          u[h][3] = uu.w;
          fv[h][0] = ff.x;
          fv[h][1] = ff.y;
          fv[h][2] = ff.z;
          fv[h][3] = ff.w;
          p1[h][0] = pp.x;
          p1[h][1] = pp.y;
          p1[h][2] = pp.z;
          p1[h][3] = pp.w;
#pragma unroll
          for (int c = 0; c < 4; ++c) {
            p2[h][c] = p2s[c];
            if (FID == FID_SEG) fv[h][c] = (fv[h][c] - A.c1) * (fv[h][c] - A.c1) - (fv[h][c] - A.c2) * (fv[h][c] - A.c2);
            if (MASK && A.mask[(size_t)(gb + br) * g.W + c0 + j0 + c]) in_d |= 1u << (4 * c + r);
          }
        }
        if (e == 0) {
          // the first row's pbar1, read by the warp above in its u-step 0
          *reinterpret_cast<float4*>(sQ1 + w * BW + j0) = make_float4(p1[0][0], p1[0][1], p1[0][2], p1[0][3]);
        }
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          float h1[2] = {p1[0][c], p1[1][c]}, h2[2] = {p2[0][c], p2[1][c]};
          if (e == 0 && i0 == 0 && s_top) h1[0] = phat_t(p1[0][c], smem[L::XLT + j0 + c], tau);
          if (c == 0 && l == 0 && s_lft) {
            h2[0] = phat_t(p2[0][0], smem[L::XLL + lr0 + e], tau);
            h2[1] = phat_t(p2[1][0], smem[L::XLL + lr0 + e + 2], tau);
          }
          U[c][e] = pk2(u[0][c], u[1][c]);
          P1[c][e] = pk2(p1[0][c], p1[1][c]);
          P2[c][e] = pk2(p2[0][c], p2[1][c]);
          H1[c][e] = pk2(h1[0], h1[1]);
          H2[c][e] = pk2(h2[0], h2[1]);
          Q1[c][e] = P1[c][e];
          Q2[c][e] = P2[c][e];
          FV[c][e] = pk2(fv[0][c], fv[1][c]);
        }
      }
#pragma unroll
      for (int c = 0; c < 4; ++c) *reinterpret_cast<ulonglong2*>(myF + c * 128) = make_ulonglong2(FV[c][0], FV[c][1]);
      *reinterpret_cast<ulonglong2*>(myQL) = make_ulonglong2(P2[0][0], P2[0][1]);
      if (last_row_here) {
        float pB[4] = {0.f, 0.f, 0.f, 0.f}, hB[4] = {0.f, 0.f, 0.f, 0.f};
        if (s_bot) {
#pragma unroll
          for (int c = 0; c < 4; ++c) {
            pB[c] = smem[L::XPB + j0 + c];
            hB[c] = phat_s(pB[c], smem[L::XLB + j0 + c], tau);
          }
        }
        const float4 pv = make_float4(pB[0], pB[1], pB[2], pB[3]);
        *reinterpret_cast<float4*>(smem + L::PBS + j0) = pv;
        *reinterpret_cast<float4*>(smem + L::HBS + j0) = make_float4(hB[0], hB[1], hB[2], hB[3]);
        *reinterpret_cast<float4*>(sQ1 + NW * BW + j0) = pv;
      }
      if (need_qh)
        *reinterpret_cast<float4*>(sQ1 + NW * BW + j0) = *reinterpret_cast<const float4*>(smem + L::XQH + j0);
      if (w == 1 && l < BAND) {
        float q = 0.f;  // an inactive right side (image boundary) reads as 0
        if (s_rgt) {
          pr_s = smem[L::SP2 + l * L::P2S + o + 128];
          hr_s = phat_s(pr_s, smem[L::XLR + l], tau);
          q = pr_s;
        }
        smem[L::QL + r_slot] = q;
      }
    }
    __syncthreads();  // staging consumed by every thread
    int nxt = cur;  // slot of the next subdomain's descriptor
    if constexpr (Src::kBatch) {
      if (t + stride < T && img_next != dsc[cur].img) {
        nxt = cur ^ 1;
        load_batch_desc(&dsc[nxt], S.B, img_next, tid, NT);
        __syncthreads();
      }
      if (t + stride < T) prefetch(t + stride, dsc[nxt].A, t + stride - dsc[nxt].base);
    } else {
      if (t + stride < T) prefetch(t + stride, S.args(t + stride), S.local(t + stride));
    }

    // unrolled by two: the new dual values then land in the registers the old ones of
    // the previous iteration held, instead of being moved back every iteration
#pragma unroll 2
    for (int k = 0; k < K; ++k) {
      const ulonglong2 cf0 = *reinterpret_cast<const ulonglong2*>(sCo + 16 * k);
      const ulonglong2 cf1 = *reinterpret_cast<const ulonglong2*>(sCo + 16 * k + 4);
      const ulonglong2 cf2 = *reinterpret_cast<const ulonglong2*>(sCo + 16 * k + 8);
      const ulonglong2 cf3 = *reinterpret_cast<const ulonglong2*>(sCo + 16 * k + 12);
      const f32x2 SIG = cf0.x, UA = cf0.y, UB = cf1.x, PA = cf2.x, PC = cf2.y, PB = cf3.x, TH = cf3.y;
      const Coef co{lo2(SIG), lo2(UA), lo2(UB), lo2(cf1.y), lo2(PA), lo2(PC), lo2(PB), lo2(TH)};
      // adaptive stop: this thread's sums of (p^{k+1} - p^k)^2 and (p^{k+1})^2 over its dofs
      f32x2 AD = 0ull, AP = 0ull;
      auto res2 = [&](f32x2 pn, f32x2 po) {
        const f32x2 d = sub2(pn, po);
        AD = fma2(d, d, AD);
        AP = fma2(pn, pn, AP);
      };
      if (ADAPT && k > 0) {
        // u of iteration k - 1 into the out-buffer: the result if the decision on iteration
        // k - 1, taken during this u-step, stops the solve
#pragma unroll
        for (int r = 0; r < 4; ++r) {
          const int e = r & 1, h = r >> 1;
          *reinterpret_cast<float4*>(smem + L::OU + (lr0 + r) * BW + j0) =
              make_float4(lane4(U[0][e], h), lane4(U[1][e], h), lane4(U[2][e], h), lane4(U[3][e], h));
        }
      }
      if (ADAPT && k > 0 && w == L::kReduceWarp) {
        // the CTA's residual sums of iteration k - 1 to every CTA of the cluster (this warp
        // then waits for the pbar1 halo anyway)
        f32x2 D = 0ull, P = 0ull;
#pragma unroll
        for (int q = 0; q < NT / 32; ++q) {
          const float4 r = *reinterpret_cast<const float4*>(smem + L::PS + 4 * (l + 32 * q));
          D = add2(D, pk2(r.x, r.y));
          P = add2(P, pk2(r.z, r.w));
        }
        f32x2 v = pk2(lo2(D) + hi2(D), lo2(P) + hi2(P));
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v = add2(v, __shfl_xor_sync(0xffffffffu, v, o));
        if (l < CL)  // lane l to CTA l, slot rank
          st_async_v2(map_rank(smem_addr(smem + L::RED + 2 * CL * (gred & 1) + 2 * rank), l), lo2(v), hi2(v),
                      map_rank(mbR + 8 * (gred & 1), l));
      }
      if (need_qh && k > 0) wait_q();  // pbar1 halo of iteration k-1
      // ---- u-step: pair e = 1 (holding the warp's last row) first
      {
        const float4 qb = *reinterpret_cast<const float4*>(sQ1 + (w + 1) * BW + j0);  // pbar1 of the row below
        // left edge of the lane to the right; lane 31 reads the slot after it, which holds
        // the tile's right side (0 when that side is on the image boundary)
        const ulonglong2 qn = *reinterpret_cast<const ulonglong2*>(myQL + 4);
        const f32x2 QRn[2] = {qn.x, qn.y};
        const float qbv[4] = {qb.x, qb.y, qb.z, qb.w};
#pragma unroll
        for (int ee = 0; ee < 2; ++ee) {
          const int e = 1 - ee;
#pragma unroll
          for (int c = 0; c < 4; ++c) {
            const ulonglong2 fc = *reinterpret_cast<const ulonglong2*>(myF + c * 128);
            const f32x2 fg = e == 0 ? fc.x : fc.y;
            // bottom - top: for e = 1 the bottom rows (2, 4) straddle pair 0 and the row
            // below, so the two lanes are subtracted as scalars straight into the pair
            const f32x2 bt = e == 0 ? sub2(Q1[c][1], Q1[c][0])
                                    : pk2(hi2(Q1[c][0]) - lo2(Q1[c][1]), qbv[c] - hi2(Q1[c][1]));
            const f32x2 right = c < 3 ? Q2[c + 1][e] : QRn[e];
            const f32x2 d = sub2(add2(bt, right), Q2[c][e]);  // div_px
            const f32x2 ub = fma2(SIG, d, U[c][e]);
            const bool dl = MASK && ((in_d >> (4 * c + e)) & 1u), dh = MASK && ((in_d >> (4 * c + e + 2)) & 1u);
            f32x2 un;
            if (FID == FID_L2) {
              un = fma2(UB, fg, mul2(UA, ub));
              if (MASK) un = pk2(dl ? lo2(ub) : lo2(un), dh ? hi2(ub) : hi2(un));
            } else {
              if (FID == FID_L1) {  // ubar - P_[-s,s](ubar - f), packed (the scalar prox_ubar's arithmetic)
                const f32x2 v = sub2(ub, fg);
                un = sub2(ub, pk2(clamp_abs(lo2(v), co.s), clamp_abs(hi2(v), co.s)));
                if (MASK) un = pk2(dl ? lo2(ub) : lo2(un), dh ? hi2(ub) : hi2(un));
              } else {
                un = pk2(prox_ubar<FID>(lo2(ub), lo2(fg), dl, co), prox_ubar<FID>(hi2(ub), hi2(fg), dh, co));
              }
            }
            U[c][e] = un;
          }
          if (e == 1 && push_down)
            st_async_v4_f32(remote_u, hi2(U[0][1]), hi2(U[1][1]), hi2(U[2][1]), hi2(U[3][1]), remote_mbU);
        }
        *reinterpret_cast<ulonglong2*>(myUR) = make_ulonglong2(U[3][0], U[3][1]);
        if (w < NW - 1)
          *reinterpret_cast<float4*>(sUB + (w + 1) * BW + j0) =
              make_float4(hi2(U[0][1]), hi2(U[1][1]), hi2(U[2][1]), hi2(U[3][1]));
        else if (last_row_here && s_bot)  // the tile's last row, for the bottom side's update
          *reinterpret_cast<float4*>(smem + L::XQH + j0) =
              make_float4(hi2(U[0][1]), hi2(U[1][1]), hi2(U[2][1]), hi2(U[3][1]));
      }
      // adaptive stop: the P1 out-buffer takes the residual sums of this iteration's p-step
      if (ADAPT && k == 0 && tid == 0) tma_wait_read();
      if (ADAPT && k > 0) {
        // decision on iteration k - 1 (eq. stop_inner1): the deciding warp adds the CL CTA
        // pairs in a fixed tree, so every CTA of the cluster takes the same decision
        if (w == L::kDecideWarp) {
          const uint32_t mb = mbR + 8 * (gred & 1);
          if (!mbar_wait(mb, (gred >> 1) & 1)) timed_out = true;
          f32x2 v = l < CL ? *reinterpret_cast<const f32x2*>(smem + L::RED + 2 * CL * (gred & 1) + 2 * l) : 0ull;
#pragma unroll
          for (int o = CL / 2; o > 0; o >>= 1) v = add2(v, __shfl_xor_sync(0xffffffffu, v, o));
          if (l == 0) {
            mbar_arrive_expect_tx(mb, L::kRedBytes);  // the barrier's next phase
            const float td = lo2(v), tp = hi2(v);
            *reinterpret_cast<int*>(smem + L::STOP) =
                (timed_out || tp == 0.f || td < (float)A.inner_tol2 * tp) ? 1 : 0;
          }
        }
        ++gred;
      }
      __syncthreads();
      if (ADAPT && k > 0 && *reinterpret_cast<const int*>(smem + L::STOP)) {
        // keep iterations 0 .. k - 1: u of iteration k - 1 waits in the out-buffer; the u
        // halo this u-step sent is drained
        k_run = k;
        if (need_uh) wait_u();
        break;
      }
      // ---- p-step: first the dofs that do not need the row above the warp (for warp 0
      // that row is the u halo from the CTA above, which is still on its way), then the
      // pbar1 of the warp's first row and its push upwards
      {
        const ulonglong2 ul = *reinterpret_cast<const ulonglong2*>(myUR - 4);  // right column of the lane to the left
#pragma unroll
        for (int e = 0; e < 2; ++e) {
#pragma unroll
          for (int c = 0; c < 4; ++c) {
            const f32x2 leftu = c > 0 ? U[c - 1][e] : (e == 0 ? ul.x : ul.y);
            if (e == 1) {
              const f32x2 tt = fma2(PC, sub2(U[c][1], U[c][0]), fma2(PA, P1[c][1], mul2(PB, H1[c][1])));  // p_target
              const f32x2 pn = pk2(clamp_abs(lo2(tt), 1.f), clamp_abs(hi2(tt), 1.f));
              Q1[c][1] = fma2(TH, sub2(pn, P1[c][1]), pn);
              if (ADAPT) res2(pn, P1[c][1]);
              P1[c][1] = pn;
            }
            {
              const f32x2 tt = fma2(PC, sub2(U[c][e], leftu), fma2(PA, P2[c][e], mul2(PB, H2[c][e])));
              const float ll = c == 0 ? lim_left : 1.f;
              const f32x2 pn = pk2(clamp_abs(lo2(tt), ll), clamp_abs(hi2(tt), ll));
              Q2[c][e] = fma2(TH, sub2(pn, P2[c][e]), pn);
              if (ADAPT) res2(pn, P2[c][e]);
              P2[c][e] = pn;
            }
          }
        }
        *reinterpret_cast<ulonglong2*>(myQL) = make_ulonglong2(Q2[0][0], Q2[0][1]);
        if (need_uh) wait_u();  // u halo of iteration k
        const float4 ua = *reinterpret_cast<const float4*>(sUB + w * BW + j0);  // u of the row above
        const float uav[4] = {ua.x, ua.y, ua.z, ua.w};
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          // u - u_above of rows (0, 2): the rows above (-1, 1) straddle the halo and pair 1
          const f32x2 du = pk2(lo2(U[c][0]) - uav[c], hi2(U[c][0]) - lo2(U[c][1]));
          const f32x2 tt = fma2(PC, du, fma2(PA, P1[c][0], mul2(PB, H1[c][0])));
          const f32x2 pn = pk2(clamp_abs(lo2(tt), lim_top), clamp_abs(hi2(tt), 1.f));
          Q1[c][0] = fma2(TH, sub2(pn, P1[c][0]), pn);
          if (ADAPT) res2(pn, P1[c][0]);
          P1[c][0] = pn;
        }
        const float4 q = make_float4(lo2(Q1[0][0]), lo2(Q1[1][0]), lo2(Q1[2][0]), lo2(Q1[3][0]));
        if (w > 0) *reinterpret_cast<float4*>(sQ1 + w * BW + j0) = q;
        if (push_up) st_async_v4_f32(remote_q1, q.x, q.y, q.z, q.w, remote_mbQ);
      }
      if (right_rows) {  // Du = -u of column 127 ((-pc) u = pc (-u) exactly)
        const float tt = fmaf(-co.pc, smem[L::UR + r_slot], fmaf(co.pa, pr_s, co.pb * hr_s));
        const float pn = clamp_abs(tt, 1.f);
        smem[L::QL + r_slot] = fmaf(co.th, pn - pr_s, pn);
        if (ADAPT) res2(pk2(pn, 0.f), pk2(pr_s, 0.f));
        pr_s = pn;
      }
      if (bottom_warp && s_bot) {  // the tile's bottom side, Du = -u of the last row
        const float4 pv = *reinterpret_cast<const float4*>(smem + L::PBS + j0);
        const float4 hv = *reinterpret_cast<const float4*>(smem + L::HBS + j0);
        const float4 uv = *reinterpret_cast<const float4*>(smem + L::XQH + j0);
        float pB[4] = {pv.x, pv.y, pv.z, pv.w}, qB[4];
        const float hB[4] = {hv.x, hv.y, hv.z, hv.w}, uB[4] = {uv.x, uv.y, uv.z, uv.w};
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          const float po = pB[c];
          p_update(pB[c], qB[c], -uB[c], hB[c], co);
          if (ADAPT) res2(pk2(pB[c], 0.f), pk2(po, 0.f));
        }
        *reinterpret_cast<float4*>(smem + L::PBS + j0) = make_float4(pB[0], pB[1], pB[2], pB[3]);
        *reinterpret_cast<float4*>(sQ1 + NW * BW + j0) = make_float4(qB[0], qB[1], qB[2], qB[3]);
      }
      if (ADAPT && k + 1 < K)  // this thread's residual sums, added up at the start of iteration k + 1
        *reinterpret_cast<float4*>(smem + L::PS + 4 * tid) = make_float4(lo2(AD), hi2(AD), lo2(AP), hi2(AP));
      if (!ADAPT && TMA && k == K - 1 && tid == 0) tma_wait_read();  // the out-buffer is free for this subdomain's bands
      __syncthreads();
    }
    const bool stopped = ADAPT && k_run < K;
    if (need_qh && !stopped) wait_q();  // drain the last pbar1 halo (not read)
    if (ADAPT && rank == 0 && tid == 0) {
      A.inner_used[t] = k_run;
      atomicMax(A.inner_max, k_run);
      atomicAdd(A.inner_work, (unsigned long long)(BW * BW) * (unsigned long long)k_run);
    }

#pragma unroll
    for (int r = 0; r < 4; ++r) {
      const int e = r & 1, h = r >> 1;
      const int gi = gb + lr0 + r;
      const float4 uv = make_float4(lane4(U[0][e], h), lane4(U[1][e], h), lane4(U[2][e], h), lane4(U[3][e], h));
      const float4 pv = make_float4(lane4(P1[0][e], h), lane4(P1[1][e], h), lane4(P1[2][e], h), lane4(P1[3][e], h));
      if (TMA) {
        if (!stopped) *reinterpret_cast<float4*>(smem + L::OU + (lr0 + r) * BW + j0) = uv;
        *reinterpret_cast<float4*>(smem + L::OP1 + (lr0 + r) * BW + j0) = pv;
      } else {
        *reinterpret_cast<float4*>(A.u + (size_t)gi * g.W + c0 + j0) = uv;
        *reinterpret_cast<float4*>(A.P1 + (size_t)(gi + a) * g.W + c0 + j0) = pv;
      }
      float* p2row = A.P2 + (size_t)gi * W2 + c0 + b + j0;
#pragma unroll
      for (int c = 0; c < 4; ++c) p2row[c] = lane4(P2[c][e], h);
      if (l == 0 && s_lft) out.SL[(size_t)(b - 1) * g.H + gi] = lane4(P2[0][e], h);
    }
    if (right_rows) {
      const int gi = gb + l;
      A.P2[(size_t)gi * W2 + c0 + 128 + b] = pr_s;
      out.SR[(size_t)b * g.H + gi] = pr_s;
    }
    if (i0 == 0 && s_top)
      *reinterpret_cast<float4*>(out.ST + (ptrdiff_t)(a - 1) * g.W + c0 + j0) =
          make_float4(lo2(P1[0][0]), lo2(P1[1][0]), lo2(P1[2][0]), lo2(P1[3][0]));
    if (last_row_here && s_bot) {
      const float4 v = *reinterpret_cast<const float4*>(smem + L::PBS + j0);
      *reinterpret_cast<float4*>(A.P1 + (size_t)(a * 128 + 128 + a) * g.W + c0 + j0) = v;
      *reinterpret_cast<float4*>(out.SB + (size_t)a * g.W + c0 + j0) = v;
    }
    if (TMA) {
      tma_fence_smem();  // the out-buffer writes become visible to the tensor stores
      pa = a;
      pc0 = c0;
      pgb = gb;
    }
    cur = nxt;
    };  // body
    if constexpr (Src::kBatch) {
      switch (dsc[cur].fid) {
        case FID_L2: body(FidC<FID_L2>{}); break;
        case FID_L1: body(FidC<FID_L1>{}); break;
        default: body(FidC<FID_SEG>{}); break;
      }
    } else {
      S.dispatch(t, body);
    }
  }
  if (TMA && pa >= 0) {  // the last subdomain's bands
    __syncthreads();
    if (tid == 0) {
      tma_store_2d(&M->u, smem + L::OU, pc0, pgb);
      tma_store_2d(&M->p1, smem + L::OP1, pc0, pgb + pa);
      tma_commit();
    }
  }
  if (TMA && tid == 0) tma_wait_all();  // the stores are complete before the CTA's shared memory is released
  cp_async_wait_all();
  cluster_arrive<true>();  // no CTA leaves while a neighbour may still write into it
  cluster_wait();
  if (timed_out) atomicOr(S.err(), 1);
}

template <int FID, bool MASK>
__global__ void __launch_bounds__(Mt4Layout::NT, 3) k_fused_mt4(const LocalArgs A) {
  fused_mt4_body<MASK, false, false>(Mt4One<FID>{A}, nullptr, blockIdx.y, gridDim.y);
}

template <int FID, bool MASK, bool ADAPT>
__global__ void __launch_bounds__(Mt4Layout::NT, 3) k_fused_mt4t(const LocalArgs A, const __grid_constant__ Mt4Maps M) {
  fused_mt4_body<MASK, true, ADAPT>(Mt4One<FID>{A}, &M, blockIdx.y, gridDim.y);
}

// the batch's work list: every subdomain with its image's descriptor and fidelity
__global__ void __launch_bounds__(Mt4Layout::NT, 3) k_fused_mt4_batch(const BatchArgs B, int total) {
  fused_mt4_body<false, false, false>(BatchTiles{B, total}, nullptr, blockIdx.y, gridDim.y);
}

// kernel kinds: cp.async copies, tensor copies, tensor copies with the adaptive stop
enum Mt4Kind { kMt4Cp = 0, kMt4Tma = 1, kMt4TmaAdapt = 2 };

// clusters of each kernel resident at once, per device: [kind][FID * 2 + MASK]
int& mt4_clusters(int dev, int kind, int fid, bool mask) {
  static int n[64][3][6] = {};
  return n[dev & 63][kind][fid * 2 + (mask ? 1 : 0)];
}

cudaLaunchConfig_t mt4_config(int clusters, bool tma, cudaLaunchAttribute* attr) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(Mt4Layout::CL, clusters, 1);
  cfg.blockDim = dim3(Mt4Layout::NT, 1, 1);
  cfg.dynamicSmemBytes = tma ? Mt4Layout::BYTES_TMA : Mt4Layout::BYTES;
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = Mt4Layout::CL;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cfg;
}

template <class Kern>
cudaError_t prepare_kernel(Kern kern, int kind, int fid, bool mask) {
  const bool tma = kind != kMt4Cp;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)(tma ? Mt4Layout::BYTES_TMA : Mt4Layout::BYTES));
  if (e != cudaSuccess) return e;
  cudaLaunchAttribute attr[1];
  cudaLaunchConfig_t cfg = mt4_config(1024, tma, attr);
  int n = 0;
  if (cudaOccupancyMaxActiveClusters(&n, kern, &cfg) != cudaSuccess) {
    cudaGetLastError();
    n = 0;
  }
  int dev = 0;
  cudaGetDevice(&dev);
  mt4_clusters(dev, kind, fid, mask) = n;
  return cudaSuccess;
}

// clusters of the batch kernel resident at once, per device
int& mt4_batch_clusters(int dev) {
  static int n[64] = {};
  return n[dev & 63];
}

// the batch kernel keeps its descriptors in the P1 out-buffer region: it is launched with
// the tensor-copy kernel's shared-memory size
static_assert(2 * sizeof(Mt4BatchDesc) <= sizeof(float) * Mt4Layout::BAND * Mt4Layout::BW &&
                  Mt4Layout::OP1 >= Mt4Layout::MB + 6,
              "two descriptors fit the P1 out-buffer, clear of the cp.async kernel's mbarriers");

cudaError_t prepare_mt4_batch() {
  cudaError_t e = cudaFuncSetAttribute(k_fused_mt4_batch, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)Mt4Layout::BYTES_TMA);
  if (e != cudaSuccess) return e;
  cudaLaunchAttribute attr[1];
  cudaLaunchConfig_t cfg = mt4_config(1024, true, attr);
  int n = 0;
  if (cudaOccupancyMaxActiveClusters(&n, k_fused_mt4_batch, &cfg) != cudaSuccess) {
    cudaGetLastError();
    n = 0;
  }
  int dev = 0;
  cudaGetDevice(&dev);
  mt4_batch_clusters(dev) = n;
  return cudaSuccess;
}

template <int FID, bool MASK>
cudaError_t prepare_mt4_one() {
  cudaError_t e = prepare_kernel(k_fused_mt4<FID, MASK>, kMt4Cp, FID, MASK);
  if (e != cudaSuccess) return e;
  if ((e = prepare_kernel(k_fused_mt4t<FID, MASK, false>, kMt4Tma, FID, MASK)) != cudaSuccess) return e;
  return prepare_kernel(k_fused_mt4t<FID, MASK, true>, kMt4TmaAdapt, FID, MASK);
}

int mt4_grid(const LocalArgs& a, int kind, int fid, bool mask) {
  int dev = 0;
  cudaGetDevice(&dev);
  const int tiles = a.g.NR * a.g.NC;
  int nc = mt4_clusters(dev, kind, fid, mask);
  return (nc <= 0 || nc > tiles) ? tiles : nc;
}

template <int FID, bool MASK>
cudaError_t launch_mt4_one(const LocalArgs& a, cudaStream_t st) {
  cudaLaunchAttribute attr[1];
  cudaLaunchConfig_t cfg = mt4_config(mt4_grid(a, kMt4Cp, FID, MASK), false, attr);
  cfg.stream = st;
  return cudaLaunchKernelEx(&cfg, k_fused_mt4<FID, MASK>, a);
}

template <int FID, bool MASK, bool ADAPT>
cudaError_t launch_mt4t_one(const LocalArgs& a, const Mt4Maps& maps, cudaStream_t st) {
  cudaLaunchAttribute attr[1];
  cudaLaunchConfig_t cfg = mt4_config(mt4_grid(a, ADAPT ? kMt4TmaAdapt : kMt4Tma, FID, MASK), true, attr);
  cfg.stream = st;
  return cudaLaunchKernelEx(&cfg, k_fused_mt4t<FID, MASK, ADAPT>, a, maps);
}

template <bool ADAPT>
cudaError_t launch_mt4t_fid(const LocalArgs& a, const Mt4Maps& maps, int fid, cudaStream_t st) {
  const bool m = a.mask != nullptr;
  switch (fid) {
    case FID_L2:
      return m ? launch_mt4t_one<FID_L2, true, ADAPT>(a, maps, st) : launch_mt4t_one<FID_L2, false, ADAPT>(a, maps, st);
    case FID_L1:
      return m ? launch_mt4t_one<FID_L1, true, ADAPT>(a, maps, st) : launch_mt4t_one<FID_L1, false, ADAPT>(a, maps, st);
    default: return launch_mt4t_one<FID_SEG, false, ADAPT>(a, maps, st);
  }
}

// cuTensorMapEncodeTiled from the driver (no link-time dependency on libcuda)
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_tiled() {
  static EncodeTiledFn fn = nullptr;
  static bool tried = false;
  if (!tried) {
    tried = true;
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(p);
    else
      cudaGetLastError();
  }
  return fn;
}

// 2-D float32 map of a rows x cols array (row pitch = cols) with boxes of box_cols x 16
bool encode_map(CUtensorMap* m, const void* base, uint64_t cols, uint64_t rows, uint32_t box_cols) {
  EncodeTiledFn fn = encode_tiled();
  if (!fn) return false;
  const cuuint64_t dim[2] = {cols, rows};
  const cuuint64_t stride[1] = {cols * sizeof(float)};
  const cuuint32_t box[2] = {box_cols, (cuuint32_t)Mt4Layout::BAND};
  const cuuint32_t es[2] = {1, 1};
  return fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<void*>(base), dim, stride, box, es,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

bool encode_maps(const LocalArgs& a, Mt4Maps* m) {
  const Grid& g = a.g;
  return encode_map(&m->u, a.u, g.W, g.H, 128) && encode_map(&m->f, a.f, g.W, g.H, 128) &&
         encode_map(&m->p1, a.P1, g.W, g.H + g.NR, 128) &&
         encode_map(&m->p2, a.P2, g.W + g.NC, g.H, Mt4Layout::P2S);
}

}  // namespace

bool fused_mt4_supported(const LocalArgs& a) {
  auto al16 = [](const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15) == 0; };
  // the inner loop reads every coefficient set from shared memory: K <= kMaxSmemCoef
  return a.K <= Mt4Layout::kMaxSmemCoef && a.g.H == 128 * a.g.NR && a.g.W == 128 * a.g.NC &&
         (a.g.W + a.g.NC) % 4 == 0 && al16(a.u) && al16(a.f) &&
         al16(a.P1) && al16(a.P2) && al16(a.lamh) && al16(a.lamv) && al16(a.out.ST) && al16(a.out.SB);
}

int fused_mt4_max_inner() { return Mt4Layout::kMaxSmemCoef; }

cudaError_t launch_fused_mt4_batch(const BatchArgs& B, int total_tiles, cudaStream_t st) {
  int dev = 0;
  cudaGetDevice(&dev);
  const int nc = mt4_batch_clusters(dev);
  cudaLaunchAttribute attr[1];
  cudaLaunchConfig_t cfg = mt4_config((nc <= 0 || nc > total_tiles) ? total_tiles : nc, true, attr);  // smem size
  cfg.stream = st;
  return cudaLaunchKernelEx(&cfg, k_fused_mt4_batch, B, total_tiles);
}

cudaError_t fused_mt4_prepare() {
  cudaError_t e;
  if ((e = prepare_mt4_batch()) != cudaSuccess) return e;
  if ((e = prepare_mt4_one<FID_L2, false>()) != cudaSuccess) return e;
  if ((e = prepare_mt4_one<FID_L2, true>()) != cudaSuccess) return e;
  if ((e = prepare_mt4_one<FID_L1, false>()) != cudaSuccess) return e;
  if ((e = prepare_mt4_one<FID_L1, true>()) != cudaSuccess) return e;
  return prepare_mt4_one<FID_SEG, false>();
}

cudaError_t launch_fused_mt4(const LocalArgs& a, int fid, bool tma, cudaStream_t st) {
  const bool m = a.mask != nullptr;
  Mt4Maps maps;
  if (a.inner_tol2 > 0.0) {  // the adaptive stop exists in the tensor-copy kernel only
    if (!encode_maps(a, &maps)) return cudaErrorNotSupported;
    return launch_mt4t_fid<true>(a, maps, fid, st);
  }
  if (tma && encode_maps(a, &maps)) return launch_mt4t_fid<false>(a, maps, fid, st);
  switch (fid) {
    case FID_L2: return m ? launch_mt4_one<FID_L2, true>(a, st) : launch_mt4_one<FID_L2, false>(a, st);
    case FID_L1: return m ? launch_mt4_one<FID_L1, true>(a, st) : launch_mt4_one<FID_L1, false>(a, st);
    default: return launch_mt4_one<FID_SEG, false>(a, st);
  }
}

}  // namespace ddtv
