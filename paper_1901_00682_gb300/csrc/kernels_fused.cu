// Fused local solver: all inner iterations of one outer iteration of Algorithm 1 for
// every subdomain in one launch (Section 5, local problem eq. local, solved by the
// accelerated primal-dual algorithm with the dual field p as the uniformly convex
// variable; projection onto the box C of eq. proj_C fused into the p-step).
//
// Mapping.  One subdomain (tile of mr x mc pixels, mc <= BW, mr <= CL*TR*R) is owned
// by a thread-block cluster of CL CTAs; CTA `rank` of the cluster owns a band of
// TR*R tile rows, and inside it thread (x, y) owns pixel column x and the R
// consecutive rows y*R .. y*R+R-1 of the band (lanes of a warp = 32 adjacent
// columns).  A thread keeps, in registers, for each of its pixels: u, the top-edge
// and left-edge dofs p1, p2 of the torn dual field, their proximal centres phat and
// extrapolations pbar, and f (or g for segmentation).  Only the values a neighbour
// needs go through shared memory: u (read by the right and lower neighbours in the
// p-step) and pbar2 (read by the left neighbour in the u-step), plus one row per
// thread row for pbar1 and u at strip ends.  Rows crossing a CTA boundary are
// pushed into the neighbour CTA's shared memory (distributed shared memory) before
// the cluster barrier.  Two barriers per inner iteration (after the u-step and after
// the p-step).  Nothing but the state load/store at the start/end of the launch
// touches global memory.
#include <cooperative_groups.h>

#include "internal.cuh"

namespace cg = cooperative_groups;

namespace ddtv {

namespace {

template <int CL>
__device__ __forceinline__ void band_sync() {
  if constexpr (CL > 1) {
    cg::this_cluster().sync();  // barrier.cluster.arrive.release + wait.acquire
  } else {
    __syncthreads();
  }
}

template <int BW, int R, int TR>
struct SmemLayout {
  static constexpr int BAND = TR * R;
  static constexpr int U = 0;                          // BAND x BW     u of the band
  static constexpr int UH = U + BAND * BW;             // BW            u of the row above the band
  static constexpr int P2 = UH + BW;                   // BAND x (BW+1) pbar2 (left edges; column mc = right side)
  static constexpr int P1 = P2 + BAND * (BW + 1);      // (TR+1) x BW   pbar1 of each thread row's first row;
                                                       //               row TR: first row of the band below
  static constexpr int PR = P1 + (TR + 1) * BW;        // BAND          right-side p
  static constexpr int HR = PR + BAND;                 // BAND          right-side phat
  static constexpr int FLOATS = HR + BAND;
  static constexpr size_t BYTES = sizeof(float) * FLOATS;
};

template <int BW, int R, int TR, int CL, int FID, bool MASK>
__global__ void __launch_bounds__(BW* TR) k_fused(const LocalArgs A) {
  using L = SmemLayout<BW, R, TR>;
  constexpr int BAND = L::BAND;
  extern __shared__ float smem[];
  float* sU = smem + L::U;
  float* sUh = smem + L::UH;
  float* sP2 = smem + L::P2;
  float* sP1 = smem + L::P1;
  float* sPR = smem + L::PR;
  float* sHR = smem + L::HR;

  const Grid g = A.g;
  const int rank = CL > 1 ? (int)blockIdx.x : 0;
  const int b = blockIdx.y, a = blockIdx.z;
  const int r0 = part_start(a, g.H, g.NR), mr = part_start(a + 1, g.H, g.NR) - r0;
  const int c0 = part_start(b, g.W, g.NC), mc = part_start(b + 1, g.W, g.NC) - c0;
  const bool s_top = a > 0, s_bot = a + 1 < g.NR, s_lft = b > 0, s_rgt = b + 1 < g.NC;
  const int j = threadIdx.x, ty = threadIdx.y;
  const int lr0 = ty * R;               // first band row of this thread
  const int i0 = rank * BAND + lr0;     // first tile row of this thread
  const bool col_ok = j < mc;
  const int W2 = g.W + g.NC;
  const int gj = c0 + j;
  const float tau = A.tau;

  float u[R], p1[R], p2[R], h1[R], h2[R], q1[R], q2[R], fg[R];
  uint32_t in_d = 0;
  float pB = 0.f, hB = 0.f, qB = 0.f;   // bottom side of the tile (thread owning row mr-1)

  // ---- load the tile's state and build the proximal centre
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const int i = i0 + r;
    u[r] = p1[r] = p2[r] = h1[r] = h2[r] = fg[r] = 0.f;
    if (col_ok && i < mr) {
      const int gi = r0 + i;
      const size_t px = (size_t)gi * g.W + gj;
      u[r] = A.u[px];
      float fv = A.f[px];
      if (FID == FID_SEG) fv = (fv - A.c1) * (fv - A.c1) - (fv - A.c2) * (fv - A.c2);
      fg[r] = fv;
      if (MASK && A.mask[px]) in_d |= 1u << r;
      p1[r] = A.P1[(size_t)(gi + a) * g.W + gj];
      p2[r] = A.P2[(size_t)gi * W2 + gj + b];
      h1[r] = (i == 0 && s_top) ? phat_t(p1[r], A.lamh[(size_t)(a - 1) * g.W + gj], tau) : p1[r];
      h2[r] = (j == 0 && s_lft) ? phat_t(p2[r], A.lamv[(size_t)(b - 1) * g.H + gi], tau) : p2[r];
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
        sP2[(lr0 + r) * (BW + 1) + mc] = pr;
      }
    }
    q1[r] = p1[r];
    q2[r] = p2[r];
    if (col_ok) sP2[(lr0 + r) * (BW + 1) + j] = q2[r];  // column mc belongs to the right side
  }
  qB = pB;
  sP1[ty * BW + j] = q1[0];
  if (CL > 1 && ty == 0 && rank > 0) {
    float* up = cg::this_cluster().map_shared_rank(sP1, rank - 1);
    up[TR * BW + j] = q1[0];
  }
  band_sync<CL>();

  // ---- inner iterations
  for (int k = 0; k < A.K; ++k) {
    const Coef c = A.coef[k];
    // u-step: u <- prox(u + sigma_k div_s pbar)
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const int i = i0 + r;
      if (col_ok && i < mr) {
        const float below = (i == mr - 1) ? qB : (r + 1 < R ? q1[r + 1] : sP1[(ty + 1) * BW + j]);
        const float right = sP2[(lr0 + r) * (BW + 1) + j + 1];
        const float d = div_px(q1[r], below, q2[r], right);
        u[r] = u_update<FID>(u[r], d, fg[r], MASK && ((in_d >> r) & 1u), c);
      }
      sU[(lr0 + r) * BW + j] = u[r];
    }
    if (CL > 1 && ty == TR - 1 && rank + 1 < CL) {
      float* dn = cg::this_cluster().map_shared_rank(sUh, rank + 1);
      dn[j] = u[R - 1];
    }
    band_sync<CL>();
    // p-step on every active dof owned by this thread
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const int i = i0 + r;
      if (col_ok && i < mr) {
        if (i > 0) {
          const float above = r > 0 ? u[r - 1] : (ty > 0 ? sU[(lr0 - 1) * BW + j] : sUh[j]);
          p_update(p1[r], q1[r], u[r] - above, h1[r], c);
        } else if (s_top) {
          p_update(p1[r], q1[r], u[r], h1[r], c);
        }
        if (j > 0) {
          p_update(p2[r], q2[r], u[r] - sU[(lr0 + r) * BW + j - 1], h2[r], c);
        } else if (s_lft) {
          p_update(p2[r], q2[r], u[r], h2[r], c);
        }
        if (i == mr - 1 && s_bot) p_update(pB, qB, -u[r], hB, c);
        if (j == mc - 1 && s_rgt) {
          float pr = sPR[lr0 + r], qr;
          p_update(pr, qr, -u[r], sHR[lr0 + r], c);
          sPR[lr0 + r] = pr;
          sP2[(lr0 + r) * (BW + 1) + mc] = qr;
        }
      }
      if (col_ok) sP2[(lr0 + r) * (BW + 1) + j] = q2[r];
    }
    sP1[ty * BW + j] = q1[0];
    if (CL > 1 && ty == 0 && rank > 0) {
      float* up = cg::this_cluster().map_shared_rank(sP1, rank - 1);
      up[TR * BW + j] = q1[0];
    }
    band_sync<CL>();
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

struct Config {
  int BW, R, TR, CL;
  const char* name;
};

// Configurations, smallest first; the first whose tile fits is used.
constexpr Config kConfigs[] = {
    {32, 8, 4, 1, "bw32_r8_tr4_cl1"},      // tiles up to 32 x 32
    {64, 8, 4, 2, "bw64_r8_tr4_cl2"},      // up to 64 x 64
    {128, 8, 2, 8, "bw128_r8_tr2_cl8"},    // up to 128 x 128
};

template <int BW, int R, int TR, int CL, int FID, bool MASK>
cudaError_t launch_one(const LocalArgs& a, cudaStream_t st) {
  using L = SmemLayout<BW, R, TR>;
  auto kern = k_fused<BW, R, TR, CL, FID, MASK>;
  // every configuration stays under the 48 KB of dynamic shared memory available
  // without an opt-in attribute, so nothing host-side is needed during graph capture
  static_assert(L::BYTES <= 48 * 1024, "fused configuration needs an opt-in shared-memory attribute");
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
  return cudaLaunchKernelEx(&cfg, kern, a);
}

template <int BW, int R, int TR, int CL>
cudaError_t launch_fid(const LocalArgs& a, int fid, cudaStream_t st) {
  const bool m = a.mask != nullptr;
  switch (fid) {
    case FID_L2: return m ? launch_one<BW, R, TR, CL, FID_L2, true>(a, st) : launch_one<BW, R, TR, CL, FID_L2, false>(a, st);
    case FID_L1: return m ? launch_one<BW, R, TR, CL, FID_L1, true>(a, st) : launch_one<BW, R, TR, CL, FID_L1, false>(a, st);
    default: return launch_one<BW, R, TR, CL, FID_SEG, false>(a, st);
  }
}

int pick(int mr, int mc) {
  for (int q = 0; q < (int)(sizeof(kConfigs) / sizeof(kConfigs[0])); ++q) {
    const Config& c = kConfigs[q];
    if (mc <= c.BW && mr <= c.R * c.TR * c.CL) return q;
  }
  return -1;
}

}  // namespace

void fused_max_tile(int* rows, int* cols) {
  const Config& c = kConfigs[sizeof(kConfigs) / sizeof(kConfigs[0]) - 1];
  *rows = c.R * c.TR * c.CL;
  *cols = c.BW;
}

const char* fused_config_name(int mr, int mc) {
  const int q = pick(mr, mc);
  return q < 0 ? "none" : kConfigs[q].name;
}

cudaError_t launch_fused_local(const LocalArgs& a, int fid, cudaStream_t st) {
  // largest tile of the (ragged) partition
  const int mr = (a.g.H + a.g.NR - 1) / a.g.NR, mc = (a.g.W + a.g.NC - 1) / a.g.NC;
  switch (pick(mr, mc)) {
    case 0: return launch_fid<32, 8, 4, 1>(a, fid, st);
    case 1: return launch_fid<64, 8, 4, 2>(a, fid, st);
    case 2: return launch_fid<128, 8, 2, 8>(a, fid, st);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace ddtv
