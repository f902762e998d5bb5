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

template <int FID, bool MASK>
__global__ void k_ustep(Grid g, float c1, float c2, const float* __restrict__ f, const uint8_t* __restrict__ mask,
                        float* __restrict__ u, const float* __restrict__ Pb1, const float* __restrict__ Pb2,
                        const Coef* __restrict__ ck) {
  const Coef c = *ck;
  const int W2 = g.W + g.NC;
  const long long n = (long long)g.H * g.W;
  for (long long px = blockIdx.x * (long long)blockDim.x + threadIdx.x; px < n;
       px += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(px / g.W), j = (int)(px % g.W);
    const int a = part_of(i, g.H, g.NR), b = part_of(j, g.W, g.NC);
    const float top = Pb1[(size_t)(i + a) * g.W + j];
    const float bot = Pb1[(size_t)(i + a + 1) * g.W + j];
    const float left = Pb2[(size_t)i * W2 + j + b];
    const float right = Pb2[(size_t)i * W2 + j + b + 1];
    float fv = f[px];
    if (FID == FID_SEG) fv = (fv - c1) * (fv - c1) - (fv - c2) * (fv - c2);
    const bool in_d = MASK && mask[px];
    u[px] = u_update<FID>(u[px], div_px(top, bot, left, right), fv, in_d, c);
  }
}

__global__ void k_pstep(Grid g, const float* __restrict__ u, float* __restrict__ P1, float* __restrict__ P2,
                        const float* __restrict__ Ph1, const float* __restrict__ Ph2, float* __restrict__ Pb1,
                        float* __restrict__ Pb2, const Coef* __restrict__ ck, int write_strips, Strips out) {
  const Coef c = *ck;
  const int W2 = g.W + g.NC;
  const long long n = (long long)g.H * g.W;
  for (long long px = blockIdx.x * (long long)blockDim.x + threadIdx.x; px < n;
       px += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(px / g.W), j = (int)(px % g.W);
    const int a = part_of(i, g.H, g.NR), b = part_of(j, g.W, g.NC);
    const int r0 = part_start(a, g.H, g.NR), r1 = part_start(a + 1, g.H, g.NR);
    const int c0 = part_start(b, g.W, g.NC), c1 = part_start(b + 1, g.W, g.NC);
    const float uc = u[px];
    // top edge of the pixel
    {
      const size_t e = (size_t)(i + a) * g.W + j;
      float p = P1[e], q;
      const float ph = Ph1 ? Ph1[e] : 0.f;
      if (i > r0) {
        p_update(p, q, uc - u[px - g.W], ph, c);
        P1[e] = p; Pb1[e] = q;
      } else if (a > 0) {
        p_update(p, q, uc, ph, c);
        P1[e] = p; Pb1[e] = q;
        if (write_strips) out.ST[(size_t)(a - 1) * g.W + j] = p;
      }
    }
    // left edge of the pixel
    {
      const size_t e = (size_t)i * W2 + j + b;
      float p = P2[e], q;
      const float ph = Ph2 ? Ph2[e] : 0.f;
      if (j > c0) {
        p_update(p, q, uc - u[px - 1], ph, c);
        P2[e] = p; Pb2[e] = q;
      } else if (b > 0) {
        p_update(p, q, uc, ph, c);
        P2[e] = p; Pb2[e] = q;
        if (write_strips) out.SL[(size_t)(b - 1) * g.H + i] = p;
      }
    }
    // bottom side of the tile
    if (i == r1 - 1 && a + 1 < g.NR) {
      const size_t e = (size_t)(i + a + 1) * g.W + j;
      float p = P1[e], q;
      p_update(p, q, -uc, Ph1 ? Ph1[e] : 0.f, c);
      P1[e] = p; Pb1[e] = q;
      if (write_strips) out.SB[(size_t)a * g.W + j] = p;
    }
    // right side of the tile
    if (j == c1 - 1 && b + 1 < g.NC) {
      const size_t e = (size_t)i * W2 + j + b + 1;
      float p = P2[e], q;
      p_update(p, q, -uc, Ph2 ? Ph2[e] : 0.f, c);
      P2[e] = p; Pb2[e] = q;
      if (write_strips) out.SR[(size_t)b * g.H + i] = p;
    }
  }
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
  const int nb = blocks_for((long long)g.H * g.W);
  const bool m = a.mask != nullptr;
  if (fid == FID_L2) {
    if (m) k_ustep<FID_L2, true><<<nb, kBlock, 0, st>>>(g, a.c1, a.c2, a.f, a.mask, a.u, Pb1, Pb2, ck);
    else k_ustep<FID_L2, false><<<nb, kBlock, 0, st>>>(g, a.c1, a.c2, a.f, a.mask, a.u, Pb1, Pb2, ck);
  } else if (fid == FID_L1) {
    if (m) k_ustep<FID_L1, true><<<nb, kBlock, 0, st>>>(g, a.c1, a.c2, a.f, a.mask, a.u, Pb1, Pb2, ck);
    else k_ustep<FID_L1, false><<<nb, kBlock, 0, st>>>(g, a.c1, a.c2, a.f, a.mask, a.u, Pb1, Pb2, ck);
  } else {
    k_ustep<FID_SEG, false><<<nb, kBlock, 0, st>>>(g, a.c1, a.c2, a.f, nullptr, a.u, Pb1, Pb2, ck);
  }
  return cudaGetLastError();
}

cudaError_t launch_plain_pstep(const LocalArgs& a, const float* Ph1, const float* Ph2, float* Pb1, float* Pb2,
                               const Coef* ck, bool write_strips, cudaStream_t st) {
  const Grid& g = a.g;
  k_pstep<<<blocks_for((long long)g.H * g.W), kBlock, 0, st>>>(g, a.u, a.P1, a.P2, Ph1, Ph2, Pb1, Pb2, ck,
                                                              write_strips ? 1 : 0, a.out);
  return cudaGetLastError();
}

}  // namespace ddtv
