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
#include <mutex>

#include "../../include/dd_tv.h"
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

// Run by every thread of the last block to finish: adds the n block partial pairs in a
// fixed order (thread t takes pairs t, t + blockDim, ...; warps, then the warp sums in
// order), so the result does not depend on scheduling and the partials' load latency
// is paid once per thread instead of once per block.
__device__ __forceinline__ void finish_pairs(const double* partials, int n, double* sj, double* sd, double& tj,
                                             double& td) {
  double a = 0.0, b = 0.0;
  for (int q = threadIdx.x; q < n; q += blockDim.x) {
    a += ((volatile const double*)partials)[2 * q];
    b += ((volatile const double*)partials)[2 * q + 1];
  }
  a = warp_sum(a);
  b = warp_sum(b);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  __syncthreads();  // the block's sj / sd are free again
  if (lane == 0) {
    sj[wid] = a;
    sd[wid] = b;
  }
  __syncthreads();
  tj = td = 0.0;
  if (threadIdx.x == 0)
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
      tj += sj[w];
      td += sd[w];
    }
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
  if (last) {
    __threadfence();
    double tj, td;
    finish_pairs(partials, (int)gridDim.x, sj, sd, tj, td);
    if (threadIdx.x == 0) {
      out[0] = tj;
      out[1] = dual ? td : -INFINITY;
      *counter = 0u;  // ready for the next call
    }
  }
}

// Primal energy only, rows of W % 4 == 0 pixels with 16-byte aligned u, f (and mask
// rows 4-byte aligned): block b takes rows b, b + gridDim.x, ...; a thread takes float4
// chunks of a row (4 pixels: their fidelity terms, the 3 differences inside the chunk,
// the one to the next chunk and the 4 to the row below).  Same compensated sums and
// fixed-order combination as k_energy, without a division per pixel.
template <int FID, bool MASK>
__global__ void __launch_bounds__(kBlock) k_energy_rows(int H, int W, float alpha, float c1, float c2,
                                                         const float* __restrict__ u, const float* __restrict__ f,
                                                         const uint8_t* __restrict__ mask,
                                                         double* __restrict__ partials,
                                                         unsigned int* __restrict__ counter, double* __restrict__ out) {
  Kahan sF, sT;
  const int W4 = W >> 2;
  for (int i = blockIdx.x; i < H; i += gridDim.x) {
    const float4* ur = reinterpret_cast<const float4*>(u + (size_t)i * W);
    const float4* fr = reinterpret_cast<const float4*>(f + (size_t)i * W);
    const bool below = i + 1 < H;
    const float4* ub = reinterpret_cast<const float4*>(u + (size_t)(i + 1) * W);
    for (int q = threadIdx.x; q < W4; q += blockDim.x) {
      const float4 a = ur[q];
      const float4 fv = fr[q];
      const float nx = q + 1 < W4 ? u[(size_t)i * W + 4 * q + 4] : a.w;
      const float4 d = below ? ub[q] : a;
      uchar4 m4 = make_uchar4(0, 0, 0, 0);
      if (MASK) m4 = reinterpret_cast<const uchar4*>(mask + (size_t)i * W)[q];
      // the chunk's terms are added in float (at most 8 non-negative terms), then once
      // into the compensated sums: short dependency chains, loads of the next chunk overlap
      const float th = (fabsf(a.y - a.x) + fabsf(a.z - a.y)) + (fabsf(a.w - a.z) + fabsf(nx - a.w));
      const float tv = (fabsf(d.x - a.x) + fabsf(d.y - a.y)) + (fabsf(d.z - a.z) + fabsf(d.w - a.w));
      sT.add(th + tv);
      const float uu[4] = {a.x, a.y, a.z, a.w}, ff[4] = {fv.x, fv.y, fv.z, fv.w};
      const unsigned char mm[4] = {m4.x, m4.y, m4.z, m4.w};
      float fe[4];
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        if (FID == FID_SEG) {
          const float gv = (ff[e] - c1) * (ff[e] - c1) - (ff[e] - c2) * (ff[e] - c2);
          fe[e] = uu[e] * gv;
        } else if (!(MASK && mm[e])) {
          const float r = uu[e] - ff[e];
          fe[e] = FID == FID_L2 ? 0.5f * r * r : fabsf(r);
        } else {
          fe[e] = 0.f;
        }
      }
      sF.add((fe[0] + fe[1]) + (fe[2] + fe[3]));
    }
  }
  double vJ = (double)alpha * ((double)sF.s - (double)sF.c) + ((double)sT.s - (double)sT.c);
  vJ = warp_sum(vJ);
  __shared__ double sj[kBlock / 32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) sj[wid] = vJ;
  __syncthreads();
  __shared__ bool last;
  if (threadIdx.x == 0) {
    double bj = 0.0;
    for (int w = 0; w < kBlock / 32; ++w) bj += sj[w];
    partials[2 * blockIdx.x] = bj;
    partials[2 * blockIdx.x + 1] = 0.0;
    __threadfence();
    const unsigned int ticket = atomicAdd(counter, 1u);
    last = ticket == gridDim.x - 1;
  }
  __syncthreads();
  if (last) {
    __threadfence();
    __shared__ double sd[kBlock / 32];
    double tj, td;
    finish_pairs(partials, (int)gridDim.x, sj, sd, tj, td);
    if (threadIdx.x == 0) {
      out[0] = tj;
      out[1] = -INFINITY;
      *counter = 0u;  // ready for the next call
    }
  }
}

// sum_j |a_j - b_j| over one row pair (the anisotropic TV across the cut between two
// row-block shards), float64, one block, fixed order
__global__ void __launch_bounds__(kBlock) k_row_tv(const float* __restrict__ a, const float* __restrict__ b, int n,
                                                   double* out) {
  __shared__ double sw[kBlock / 32];
  double v = 0.0;
  for (int j = threadIdx.x; j < n; j += kBlock) v += fabs((double)a[j] - (double)b[j]);
  v = warp_sum(v);
  if ((threadIdx.x & 31) == 0) sw[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < kBlock / 32; ++w) t += sw[w];
    *out = t;
  }
}

}  // namespace

cudaError_t launch_row_tv(const float* a, const float* b, int n, double* out, cudaStream_t st) {
  k_row_tv<<<1, kBlock, 0, st>>>(a, b, n, out);
  return cudaGetLastError();
}

int reduce_partials_count() { return 2 * kBlocks; }

cudaError_t launch_energy(const Grid& g, int fid, float alpha, float c1, float c2, const float* u, const float* f,
                          const uint8_t* mask, const float* P1, const float* P2, double* partials,
                          unsigned int* counter, double* out, cudaStream_t st) {
  const bool rows = P1 == nullptr && g.W % 4 == 0 && ((uintptr_t)u % 16 == 0) && ((uintptr_t)f % 16 == 0) &&
                    (mask == nullptr || (uintptr_t)mask % 4 == 0);
  if (!rows) {
    k_energy<<<kBlocks, kBlock, 0, st>>>(g, fid, alpha, c1, c2, u, f, mask, P1, P2, partials, counter, out);
    return cudaGetLastError();
  }
  const int nb = g.H < kBlocks ? g.H : kBlocks;
#define ROWS(F, M) k_energy_rows<F, M><<<nb, kBlock, 0, st>>>(g.H, g.W, alpha, c1, c2, u, f, mask, partials, counter, out)
  if (fid == FID_SEG) ROWS(FID_SEG, false);
  else if (fid == FID_L1) { if (mask) ROWS(FID_L1, true); else ROWS(FID_L1, false); }
  else { if (mask) ROWS(FID_L2, true); else ROWS(FID_L2, false); }
#undef ROWS
  return cudaGetLastError();
}

}  // namespace ddtv

// ---------------------------------------------------------------------------
// Energy without any allocation.
//
// The handle-based dd_tv_energy keeps its block partials in memory the handle
// allocated with cudaMalloc.  Some callers cannot allocate device memory when they
// need an energy value: a process whose device memory is entirely reserved by
// another framework's pool, or a latency-critical loop where cudaMalloc's implicit
// device synchronisation is not acceptable.  dd_tv_energy_noalloc serves them with
// the same reduction kernel, its scratch living in the file-scope array below.
//
// Scratch: kNoAllocDoubles doubles (9,760 bytes) per GPU that loads the library,
// held until the process exits: 2 partial sums per block of the fixed 608-block
// grid, the block counter, and the two results.  Because the grid never grows,
// every image up to 2^31 - 1 pixels fits; larger ones are refused.
namespace {

constexpr int kNoAllocDoubles = 2 * 152 * 4 + 4;
constexpr int kMaxDevices = 64;
static __device__ __align__(256) double g_energy_scratch[kNoAllocDoubles];

std::mutex g_scratch_mu;
double* g_scratch_ptr[kMaxDevices] = {nullptr};

// Device address of the scratch array on the current device.  In host code the
// array's name is only a host-side stand-in, so the address is looked up once per
// device with that device current (the first call on each device does this).
cudaError_t scratch_on_current_device(double** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lk(g_scratch_mu);
  if (!g_scratch_ptr[dev]) {
    double* p = nullptr;
    e = cudaGetSymbolAddress((void**)&p, g_energy_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_ptr[dev] = p;
  }
  *out = g_scratch_ptr[dev];
  return cudaSuccess;
}

}  // namespace

extern "C" int dd_tv_energy_noalloc(const float* u_dev, const float* f_dev, const uint8_t* mask_dev, int height,
                                    int width, int fidelity, double alpha, double c1, double c2, void* stream,
                                    double* J_out) {
  if (!u_dev || !f_dev || !J_out) return DD_TV_EINVAL;
  if (height < 1 || width < 1) return DD_TV_EINVAL;
  if ((long long)height * width > (1LL << 31) - 1) return DD_TV_EINVAL;  // beyond what the scratch serves
  if (fidelity < DD_TV_L2 || fidelity > DD_TV_SEG || !(alpha > 0.0)) return DD_TV_EINVAL;
  if (ddtv::reduce_partials_count() + 4 > kNoAllocDoubles) return DD_TV_EUNSUPPORTED;
  double* scratch = nullptr;
  if (scratch_on_current_device(&scratch) != cudaSuccess) return DD_TV_ECUDA;
  const cudaStream_t st = (cudaStream_t)stream;
  const int np = ddtv::reduce_partials_count();
  double* partials = scratch;
  unsigned int* counter = reinterpret_cast<unsigned int*>(scratch + np);
  double* out = scratch + np + 2;
  // the array keeps the previous call's contents: the block counter must start at 0
  if (cudaMemsetAsync(counter, 0, sizeof(unsigned int), st) != cudaSuccess) return DD_TV_ECUDA;
  const ddtv::Grid g{height, width, 1, 1};
  if (ddtv::launch_energy(g, fidelity, (float)alpha, (float)c1, (float)c2, u_dev, f_dev, mask_dev, nullptr, nullptr,
                          partials, counter, out, st) != cudaSuccess)
    return DD_TV_ECUDA;
  double host[1];
  if (cudaMemcpyAsync(host, out, sizeof(double), cudaMemcpyDeviceToHost, st) != cudaSuccess) return DD_TV_ECUDA;
  if (cudaStreamSynchronize(st) != cudaSuccess) return DD_TV_ECUDA;
  *J_out = host[0];
  return DD_TV_OK;
}
