// State initialisation: u^0 = f (with f := 0 on the inpainting domain D, Section 3)
// for the L2/L1 fidelities and u^0 = 1/2 for segmentation; and the probe of the
// bounded device-side wait (failure detection, no counterpart in the paper).
#include "fused_common.cuh"
#include "internal.cuh"

namespace ddtv {

namespace {

__global__ void k_init_u(long long n, int fid, const float* __restrict__ f, const uint8_t* __restrict__ mask,
                         float* __restrict__ u) {
  for (long long px = blockIdx.x * (long long)blockDim.x + threadIdx.x; px < n;
       px += (long long)gridDim.x * blockDim.x) {
    float v = fid == FID_SEG ? 0.5f : f[px];
    if (fid != FID_SEG && mask && mask[px]) v = 0.0f;
    u[px] = v;
  }
}

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
  return t;
}

// One thread waits, with the bounded wait of the fused kernels, on an mbarrier of its
// own CTA whose phase 0 nothing completes (one arrival expected, none made, no copy
// counted on it); when the bound runs out it sets *err as those kernels do.
__global__ void k_wait_probe(int* err, unsigned long long* waited_ns) {
  __shared__ __align__(8) unsigned long long bar;
  const uint32_t a = smem_addr(&bar);
  mbar_init(a, 1);
  const unsigned long long t0 = global_ns();
  const bool ok = mbar_wait(a, 0);
  *waited_ns = global_ns() - t0;
  if (!ok) atomicOr(err, 1);
}

}  // namespace

cudaError_t launch_wait_probe(int* err, unsigned long long* waited_ns, cudaStream_t st) {
  k_wait_probe<<<1, 1, 0, st>>>(err, waited_ns);
  return cudaGetLastError();
}

cudaError_t launch_init_u(const Grid& g, int fid, const float* f, const uint8_t* mask, float* u, cudaStream_t st) {
  const long long n = (long long)g.H * g.W;
  long long nb = (n + 255) / 256;
  if (nb > 152 * 32) nb = 152 * 32;
  k_init_u<<<(int)nb, 256, 0, st>>>(n, fid, f, mask, u);
  return cudaGetLastError();
}

}  // namespace ddtv
