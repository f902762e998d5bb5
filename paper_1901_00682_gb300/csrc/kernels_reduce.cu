// Energy and duality-gap reduction (Section 3, eq. model; stopping rule eq. stop_outer):
//   J(u) = alpha F(u) + TV(u),  TV(u) = sum |u_{i+1,j} - u_ij| + |u_{i,j+1} - u_ij|,
// and the dual value of the averaged torn field p (the two copies of an interface dof
// averaged; the average of two points of the box C is in C):
//   L2, no mask : d(p) = sum_T -(div p + alpha f)^2 / (2 alpha) + alpha f^2 / 2
//   SEG         : d(p) = sum_T min(0, alpha g - div p)
// Each thread sums its pixels in float32 with Kahan compensation, threads and blocks
// are combined in float64, and the last block to finish adds the block partials in a
// fixed order, so the result does not depend on scheduling.  HBM-bound: u, f (and
// mask, P1, P2) are read once.
#include "internal.cuh"

namespace ddtv {

namespace {

constexpr int kBlock = 256;
constexpr int kBlocks = 152 * 4;

struct Kahan {
  float s = 0.f, c = 0.f;
  __device__ __forceinline__ void add(float x) {
    const float y = x - c;
    const float t = s + y;
    c = (t - s) - y;
    s = t;
  }
};

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

// averaged global dof of the horizontal edge above pixel row i (0 < i < H), column j
__device__ __forceinline__ float avg_p1(const Grid& g, const float* P1, int i, int j) {
  const int a = part_of(i, g.H, g.NR);
  const float v = P1[(size_t)(i + a) * g.W + j];
  if (i == part_start(a, g.H, g.NR)) return 0.5f * (v + P1[(size_t)(i + a - 1) * g.W + j]);
  return v;
}

__device__ __forceinline__ float avg_p2(const Grid& g, const float* P2, int i, int l) {
  const int b = part_of(l, g.W, g.NC);
  const int W2 = g.W + g.NC;
  const float v = P2[(size_t)i * W2 + l + b];
  if (l == part_start(b, g.W, g.NC)) return 0.5f * (v + P2[(size_t)i * W2 + l + b - 1]);
  return v;
}

__global__ void __launch_bounds__(kBlock) k_energy(Grid g, int fid, float alpha, float c1, float c2,
                                                   const float* __restrict__ u, const float* __restrict__ f,
                                                   const uint8_t* __restrict__ mask, const float* __restrict__ P1,
                                                   const float* __restrict__ P2, double* __restrict__ partials,
                                                   unsigned int* __restrict__ counter, double* __restrict__ out) {
  Kahan sF, sT, sD;
  const long long n = (long long)g.H * g.W;
  const bool dual = P1 != nullptr;
  for (long long px = blockIdx.x * (long long)blockDim.x + threadIdx.x; px < n;
       px += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(px / g.W), j = (int)(px % g.W);
    const float uc = u[px];
    if (i + 1 < g.H) sT.add(fabsf(u[px + g.W] - uc));
    if (j + 1 < g.W) sT.add(fabsf(u[px + 1] - uc));
    const float fv = f[px];
    const bool in_d = mask && mask[px];
    float gv = 0.f;
    if (fid == FID_SEG) {
      gv = (fv - c1) * (fv - c1) - (fv - c2) * (fv - c2);
      sF.add(uc * gv);
    } else if (!in_d) {
      const float r = uc - fv;
      sF.add(fid == FID_L2 ? 0.5f * r * r : fabsf(r));
    }
    if (dual) {
      const float top = i > 0 ? avg_p1(g, P1, i, j) : 0.f;
      const float bot = i + 1 < g.H ? avg_p1(g, P1, i + 1, j) : 0.f;
      const float left = j > 0 ? avg_p2(g, P2, i, j) : 0.f;
      const float right = j + 1 < g.W ? avg_p2(g, P2, i, j + 1) : 0.f;
      const float d = div_px(top, bot, left, right);
      if (fid == FID_SEG) {
        sD.add(fminf(0.f, alpha * gv - d));
      } else {
        const float t = d + alpha * fv;
        sD.add(-t * t / (2.f * alpha) + 0.5f * alpha * fv * fv);
      }
    }
  }
  double vJ = (double)alpha * ((double)sF.s - (double)sF.c) + ((double)sT.s - (double)sT.c);
  double vD = (double)sD.s - (double)sD.c;
  vJ = warp_sum(vJ);
  vD = warp_sum(vD);
  __shared__ double sj[kBlock / 32], sd[kBlock / 32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) { sj[wid] = vJ; sd[wid] = vD; }
  __syncthreads();
  __shared__ bool last;
  if (threadIdx.x == 0) {
    double bj = 0.0, bd = 0.0;
    for (int w = 0; w < kBlock / 32; ++w) { bj += sj[w]; bd += sd[w]; }
    partials[2 * blockIdx.x] = bj;
    partials[2 * blockIdx.x + 1] = bd;
    __threadfence();
    const unsigned int ticket = atomicAdd(counter, 1u);
    last = ticket == gridDim.x - 1;
  }
  __syncthreads();
  if (last && threadIdx.x == 0) {
    __threadfence();
    double tj = 0.0, td = 0.0;
    for (int q = 0; q < (int)gridDim.x; ++q) {
      tj += ((volatile double*)partials)[2 * q];
      td += ((volatile double*)partials)[2 * q + 1];
    }
    out[0] = tj;
    out[1] = dual ? td : -INFINITY;
    *counter = 0u;  // ready for the next call
  }
}

}  // namespace

int reduce_partials_count() { return 2 * kBlocks; }

cudaError_t launch_energy(const Grid& g, int fid, float alpha, float c1, float c2, const float* u, const float* f,
                          const uint8_t* mask, const float* P1, const float* P2, double* partials,
                          unsigned int* counter, double* out, cudaStream_t st) {
  k_energy<<<kBlocks, kBlock, 0, st>>>(g, fid, alpha, c1, c2, u, f, mask, P1, P2, partials, counter, out);
  return cudaGetLastError();
}

}  // namespace ddtv
