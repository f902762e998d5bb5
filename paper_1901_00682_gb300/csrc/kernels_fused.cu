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
// The local solve of tile (a, b) of the problem A, its interface strips written to out.
template <int BW, int R, int TR, int CL, int FID, bool MASK, bool ADAPT>
__device__ __forceinline__ void fused_tile(const LocalArgs& A, const Strips out, const int a, const int b) {
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
  const int r0 = part_start(a, g.H, g.NR), mr = part_start(a + 1, g.H, g.NR) - r0;
  const int c0 = part_start(b, g.W, g.NC), mc = part_start(b + 1, g.W, g.NC) - c0;
  const bool s_top = a > 0 || g.cut_top, s_bot = a + 1 < g.NR || g.cut_bot, s_lft = b > 0, s_rgt = b + 1 < g.NC;
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
      b1 = (i == 0 && s_top) ? phat_t(a1, A.lamh[(ptrdiff_t)(a - 1) * g.W + gj], tau) : a1;
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
      if (i == 0 && s_top) out.ST[(ptrdiff_t)(a - 1) * g.W + gj] = p1[r];
      if (j == 0 && s_lft) out.SL[(size_t)(b - 1) * g.H + gi] = p2[r];
      if (i == mr - 1 && s_bot) {
        A.P1[(size_t)(gi + a + 1) * g.W + gj] = pB;
        out.SB[(size_t)a * g.W + gj] = pB;
      }
      if (j == mc - 1 && s_rgt) {
        const float pr = sPR[lr0 + r];
        A.P2[(size_t)gi * W2 + gj + b + 1] = pr;
        out.SR[(size_t)b * g.H + gi] = pr;
      }
    }
  }
}


template <int BW, int R, int TR, int CL, int FID, bool MASK, bool ADAPT>
__global__ void __launch_bounds__(BW* TR, (BW * TR <= 256 ? 2 : 1)) k_fused(const LocalArgs A) {
  fused_tile<BW, R, TR, CL, FID, MASK, ADAPT>(A, A.out, (int)blockIdx.z, (int)blockIdx.y);
}

// Every tile of a batch of images, one CTA cluster per tile (blockIdx.y = the batch's
// tile), each with its image's fidelity, parameters and strips.
template <int BW, int R, int TR, int CL>
__global__ void __launch_bounds__(BW* TR, (BW * TR <= 256 ? 2 : 1)) k_fused_tile_batch(const BatchArgs B) {
  const int t = blockIdx.y;
  const int img = B.tile_img[t];
  const LocalArgs A = B.args[img];
  const int q = t - B.tile_base[img];
  const int a = q / A.g.NC, b = q - a * A.g.NC;
  const Strips out = B.strips[2 * img + B.write_set];
  switch (B.fid[img]) {
    case FID_L2: fused_tile<BW, R, TR, CL, FID_L2, false, false>(A, out, a, b); break;
    case FID_L1: fused_tile<BW, R, TR, CL, FID_L1, false, false>(A, out, a, b); break;
    default: fused_tile<BW, R, TR, CL, FID_SEG, false, false>(A, out, a, b); break;
  }
}

struct Config {
  int BW, R, TR, CL;
  const char* name;
};

// Cluster-barrier mappings by tile size.  Class 0: tiles up to 32 x 32; class 1: up
// to 64 x 64; class 2: up to 128 x 128.
constexpr Config kConfigs[] = {
    {32, 8, 4, 1, "bw32_r8_tr4_cl1"},    // class 0
    {64, 8, 8, 1, "bw64_r8_tr8_cl1"},    // class 1
    {128, 8, 2, 8, "bw128_r8_tr2_cl8"},  // class 2: 256 threads, 2 CTAs/SM
};

// Hardware mappings of exact 128 x 128 subdomains (dd_tv_params.variant):
//   0  persistent 4 x 4 micro-tiles, state moved by tensor copies (default)
//   1  the same kernel moving the state with 16-byte cp.async copies
//   2  persistent 2 x 4 micro-tiles, 256 threads, 2 CTAs per SM
//   3  the cluster-barrier kernel of every other tile shape (one subdomain per cluster)
constexpr int kNumVariants = 4;

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

// index into kConfigs for a tile shape, -1 if none fits
int pick(int mr, int mc) {
  if (mc <= 32 && mr <= 32) return 0;
  if (mc <= 64 && mr <= 64) return 1;
  if (mc <= 128 && mr <= 128) return 2;
  return -1;
}

}  // namespace

void fused_max_tile(int* rows, int* cols) {
  *rows = 128;
  *cols = 128;
}

int fused_num_variants() { return kNumVariants; }

const char* fused_config_name(int mr, int mc, int variant) {
  if (mr == 128 && mc == 128) {
    switch (variant) {
      case 0: return "mt4_tma";
      case 1: return "mt4_cp_async";
      case 2: return "mt2x4";
      default: break;
    }
  }
  const int q = pick(mr, mc);
  return q < 0 ? "none" : kConfigs[q].name;
}

cudaError_t fused_prepare() {
  cudaError_t e;
  if ((e = prepare_fid<32, 8, 4, 1>()) != cudaSuccess) return e;
  if ((e = prepare_fid<64, 8, 8, 1>()) != cudaSuccess) return e;
  if ((e = cudaFuncSetAttribute(k_fused_tile_batch<64, 8, 8, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)SmemLayout<64, 8, 8>::BYTES)) != cudaSuccess)
    return e;
  if ((e = prepare_fid<128, 8, 2, 8>()) != cudaSuccess) return e;
  if ((e = fused_mt_prepare()) != cudaSuccess) return e;
  return fused_mt4_prepare();
}

cudaError_t launch_fused_batch(const BatchArgs& B, int total_tiles, int tile, int variant, int K, cudaStream_t st) {
  if (tile == 128)  // variant 0: 4 x 4 micro-tiles (K within its shared coefficient table); 2: 2 x 4
    return variant == 0 && K <= fused_mt4_max_inner() ? launch_fused_mt4_batch(B, total_tiles, st)
                                                       : launch_fused_mt_batch(B, total_tiles, st);
  if (tile != 64) return cudaErrorInvalidValue;
  // 64 x 64 subdomains: one CTA of 64 x 8 threads per subdomain
  k_fused_tile_batch<64, 8, 8, 1><<<dim3(1, total_tiles, 1), dim3(64, 8, 1), SmemLayout<64, 8, 8>::BYTES, st>>>(B);
  return cudaGetLastError();
}

cudaError_t launch_fused_local(const LocalArgs& a, int fid, int variant, cudaStream_t st) {
  // largest tile of the (ragged) partition
  const int mr = (a.g.H + a.g.NR - 1) / a.g.NR, mc = (a.g.W + a.g.NC - 1) / a.g.NC;
  const bool exact128 = a.g.H == 128 * a.g.NR && a.g.W == 128 * a.g.NC;  // every tile exactly 128 x 128
  if (a.inner_tol2 > 0.0 && exact128 && variant == 0 && fused_mt4_supported(a)) {
    // adaptive inner stop in the default kernel (the other variants: the cluster-barrier kernel)
    const cudaError_t e = launch_fused_mt4(a, fid, true, st);
    if (e != cudaErrorNotSupported) return e;
  }
  if (a.inner_tol2 <= 0.0 && exact128) {
    switch (variant) {
      case 0:  // default: persistent 4 x 4 micro-tiles, tensor copies
      case 1:  // the same with cp.async copies
        if (fused_mt4_supported(a)) return launch_fused_mt4(a, fid, variant == 0, st);
        if (fused_mt_supported(a)) return launch_fused_mt(a, fid, st);  // W + N_c not a multiple of 4
        break;
      case 2:
        if (fused_mt_supported(a)) return launch_fused_mt(a, fid, st);
        break;
      default: break;
    }
  }
  switch (pick(mr, mc)) {
    case 0: return launch_fid<32, 8, 4, 1>(a, fid, st);
    case 1: return launch_fid<64, 8, 8, 1>(a, fid, st);
    case 2: return launch_fid<128, 8, 2, 8>(a, fid, st);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace ddtv
