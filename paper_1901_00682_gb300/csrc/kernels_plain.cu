// Plain (unfused) path: one global-memory kernel per step of the local iteration,
// over all tiles at once.  It runs the same arithmetic as the fused kernel (shared
// pointwise functions, same operand order), so both paths give identical bits; it
// is the comparator for the fused path and, with a 1 x 1 grid and no proximal term,
// the full-dimension primal-dual iteration (the N = 1 comparator of Section 5).
// Every step streams its whole state through HBM.
#include "internal.cuh"

namespace ddtv {

namespace {

constexpr int kBlock = 256;

// phat <- p~ (copy) then -+ tau lambda on the interface sides; pbar <- p~
__global__ void k_phat_sides(Grid g, float tau, const float* __restrict__ P1, const float* __restrict__ P2,
                             const float* __restrict__ lamh, const float* __restrict__ lamv, float* __restrict__ Ph1,
                             float* __restrict__ Ph2) {
  const int nh = (g.NR - 1) * g.W, nv = (g.NC - 1) * g.H;
  const int W2 = g.W + g.NC;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < nh + nv; e += gridDim.x * blockDim.x) {
    if (e < nh) {
      const int a = e / g.W, j = e % g.W;
      const int rs = part_start(a + 1, g.H, g.NR) + a;
      const float lam = lamh[e];
      Ph1[(size_t)rs * g.W + j] = phat_s(P1[(size_t)rs * g.W + j], lam, tau);
      Ph1[(size_t)(rs + 1) * g.W + j] = phat_t(P1[(size_t)(rs + 1) * g.W + j], lam, tau);
    } else {
      const int q = e - nh, b = q / g.H, i = q % g.H;
      const int cs = part_start(b + 1, g.W, g.NC) + b;
      const float lam = lamv[q];
      Ph2[(size_t)i * W2 + cs] = phat_s(P2[(size_t)i * W2 + cs], lam, tau);
      Ph2[(size_t)i * W2 + cs + 1] = phat_t(P2[(size_t)i * W2 + cs + 1], lam, tau);
    }
  }
}

// Both step kernels run on a 2-D grid: blockIdx.x = (tile column b, 128-column segment
// of it), blockIdx.y strides over the pixel rows.  The tile geometry is computed once
// per block and row (no division per pixel); threads of a block read consecutive
// columns of one row of every array (coalesced).
constexpr int kSeg = 128;

struct RowCol {
  int a, r0, r1;   // tile row of the pixel row and its first / end row
  int b, c0, c1;   // tile column of the block and its first / end column
};

__device__ __forceinline__ RowCol geometry(const Grid& g, int i, int spt) {
  RowCol q;
  q.a = part_of(i, g.H, g.NR);
  q.r0 = part_start(q.a, g.H, g.NR);
  q.r1 = part_start(q.a + 1, g.H, g.NR);
  q.b = (int)blockIdx.x / spt;
  q.c0 = part_start(q.b, g.W, g.NC);
  q.c1 = part_start(q.b + 1, g.W, g.NC);
  return q;
}

template <int FID, bool MASK>
__global__ void __launch_bounds__(kSeg) k_ustep(Grid g, int spt, float c1, float c2, const float* __restrict__ f,
                                                const uint8_t* __restrict__ mask, float* __restrict__ u,
                                                const float* __restrict__ Pb1, const float* __restrict__ Pb2,
                                                const Coef* __restrict__ ck) {
  const Coef c = *ck;
  const int W2 = g.W + g.NC;
  for (int i = blockIdx.y; i < g.H; i += gridDim.y) {
    const RowCol q = geometry(g, i, spt);
    const int j = q.c0 + ((int)blockIdx.x - q.b * spt) * kSeg + (int)threadIdx.x;
    if (j >= q.c1) continue;
    const size_t px = (size_t)i * g.W + j;
    const float top = Pb1[(size_t)(i + q.a) * g.W + j];
    const float bot = Pb1[(size_t)(i + q.a + 1) * g.W + j];
    const float left = Pb2[(size_t)i * W2 + j + q.b];
    const float right = Pb2[(size_t)i * W2 + j + q.b + 1];
    float fv = f[px];
    if (FID == FID_SEG) fv = (fv - c1) * (fv - c1) - (fv - c2) * (fv - c2);
    const bool in_d = MASK && mask[px];
    u[px] = u_update<FID>(u[px], div_px(top, bot, left, right), fv, in_d, c);
  }
}

__global__ void __launch_bounds__(kSeg) k_pstep(Grid g, int spt, const float* __restrict__ u, float* __restrict__ P1,
                                                float* __restrict__ P2, const float* __restrict__ Ph1,
                                                const float* __restrict__ Ph2, float* __restrict__ Pb1,
                                                float* __restrict__ Pb2, const Coef* __restrict__ ck,
                                                int write_strips, Strips out) {
  const Coef c = *ck;
  const int W2 = g.W + g.NC;
  for (int i = blockIdx.y; i < g.H; i += gridDim.y) {
    const RowCol q = geometry(g, i, spt);
    const int a = q.a, b = q.b;
    const int j = q.c0 + ((int)blockIdx.x - b * spt) * kSeg + (int)threadIdx.x;
    if (j >= q.c1) continue;
    const size_t px = (size_t)i * g.W + j;
    const float uc = u[px];
    // top edge of the pixel
    {
      const size_t e = (size_t)(i + a) * g.W + j;
      float p = P1[e], pb;
      const float ph = Ph1 ? Ph1[e] : 0.f;
      if (i > q.r0) {
        p_update(p, pb, uc - u[px - g.W], ph, c);
        P1[e] = p; Pb1[e] = pb;
      } else if (a > 0) {
        p_update(p, pb, uc, ph, c);
        P1[e] = p; Pb1[e] = pb;
        if (write_strips) out.ST[(size_t)(a - 1) * g.W + j] = p;
      }
    }
    // left edge of the pixel
    {
      const size_t e = (size_t)i * W2 + j + b;
      float p = P2[e], pb;
      const float ph = Ph2 ? Ph2[e] : 0.f;
      if (j > q.c0) {
        p_update(p, pb, uc - u[px - 1], ph, c);
        P2[e] = p; Pb2[e] = pb;
      } else if (b > 0) {
        p_update(p, pb, uc, ph, c);
        P2[e] = p; Pb2[e] = pb;
        if (write_strips) out.SL[(size_t)(b - 1) * g.H + i] = p;
      }
    }
    // bottom side of the tile
    if (i == q.r1 - 1 && a + 1 < g.NR) {
      const size_t e = (size_t)(i + a + 1) * g.W + j;
      float p = P1[e], pb;
      p_update(p, pb, -uc, Ph1 ? Ph1[e] : 0.f, c);
      P1[e] = p; Pb1[e] = pb;
      if (write_strips) out.SB[(size_t)a * g.W + j] = p;
    }
    // right side of the tile
    if (j == q.c1 - 1 && b + 1 < g.NC) {
      const size_t e = (size_t)i * W2 + j + b + 1;
      float p = P2[e], pb;
      p_update(p, pb, -uc, Ph2 ? Ph2[e] : 0.f, c);
      P2[e] = p; Pb2[e] = pb;
      if (write_strips) out.SR[(size_t)b * g.H + i] = p;
    }
  }
}

// 2-D grid of the step kernels: (tile columns x 128-column segments of the widest tile
// column, pixel rows up to 65535, striding beyond)
struct StepGrid {
  dim3 grid;
  int spt;
};

StepGrid step_grid(const Grid& g) {
  const int wmax = (g.W + g.NC - 1) / g.NC;  // widest tile column of the partition
  StepGrid s;
  s.spt = (wmax + kSeg - 1) / kSeg;
  // about 16 blocks of 128 threads per SM, each striding over many rows (a block per
  // row segment would spend the kernel on block scheduling)
  const long long gx = (long long)g.NC * s.spt;
  long long gy = (152LL * 16 + gx - 1) / gx;
  if (gy > g.H) gy = g.H;
  if (gy > 65535) gy = 65535;
  s.grid = dim3((unsigned)gx, (unsigned)(gy < 1 ? 1 : gy), 1);
  return s;
}

int blocks_for(long long n) {
  long long b = (n + kBlock - 1) / kBlock;
  if (b > 152 * 32) b = 152 * 32;
  return (int)(b < 1 ? 1 : b);
}

}  // namespace

cudaError_t launch_plain_phat(const LocalArgs& a, float* Ph1, float* Ph2, float* Pb1, float* Pb2, cudaStream_t st) {
  const Grid& g = a.g;
  const size_t n1 = (size_t)(g.H + g.NR) * g.W, n2 = (size_t)g.H * (g.W + g.NC);
  cudaError_t e;
  if ((e = cudaMemcpyAsync(Ph1, a.P1, n1 * sizeof(float), cudaMemcpyDeviceToDevice, st)) != cudaSuccess) return e;
  if ((e = cudaMemcpyAsync(Ph2, a.P2, n2 * sizeof(float), cudaMemcpyDeviceToDevice, st)) != cudaSuccess) return e;
  if ((e = cudaMemcpyAsync(Pb1, a.P1, n1 * sizeof(float), cudaMemcpyDeviceToDevice, st)) != cudaSuccess) return e;
  if ((e = cudaMemcpyAsync(Pb2, a.P2, n2 * sizeof(float), cudaMemcpyDeviceToDevice, st)) != cudaSuccess) return e;
  const int n = (g.NR - 1) * g.W + (g.NC - 1) * g.H;
  if (n > 0) k_phat_sides<<<blocks_for(n), kBlock, 0, st>>>(g, a.tau, a.P1, a.P2, a.lamh, a.lamv, Ph1, Ph2);
  return cudaGetLastError();
}

cudaError_t launch_plain_ustep(const LocalArgs& a, const float* Pb1, const float* Pb2, const Coef* ck, int fid,
                               cudaStream_t st) {
  const Grid& g = a.g;
  const StepGrid sg = step_grid(g);
  const bool m = a.mask != nullptr;
#define USTEP(F, M) k_ustep<F, M><<<sg.grid, kSeg, 0, st>>>(g, sg.spt, a.c1, a.c2, a.f, a.mask, a.u, Pb1, Pb2, ck)
  if (fid == FID_L2) {
    if (m) USTEP(FID_L2, true); else USTEP(FID_L2, false);
  } else if (fid == FID_L1) {
    if (m) USTEP(FID_L1, true); else USTEP(FID_L1, false);
  } else {
    USTEP(FID_SEG, false);
  }
#undef USTEP
  return cudaGetLastError();
}

cudaError_t launch_plain_pstep(const LocalArgs& a, const float* Ph1, const float* Ph2, float* Pb1, float* Pb2,
                               const Coef* ck, bool write_strips, cudaStream_t st) {
  const Grid& g = a.g;
  const StepGrid sg = step_grid(g);
  k_pstep<<<sg.grid, kSeg, 0, st>>>(g, sg.spt, a.u, a.P1, a.P2, Ph1, Ph2, Pb1, Pb2, ck, write_strips ? 1 : 0, a.out);
  return cudaGetLastError();
}

}  // namespace ddtv
