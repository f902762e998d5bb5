// State initialisation: u^0 = f (with f := 0 on the inpainting domain D, Section 3)
// for the L2/L1 fidelities and u^0 = 1/2 for segmentation.
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

}  // namespace

cudaError_t launch_init_u(const Grid& g, int fid, const float* f, const uint8_t* mask, float* u, cudaStream_t st) {
  const long long n = (long long)g.H * g.W;
  long long nb = (n + 255) / 256;
  if (nb > 152 * 32) nb = 152 * 32;
  k_init_u<<<(int)nb, 256, 0, st>>>(n, fid, f, mask, u);
  return cudaGetLastError();
}

}  // namespace ddtv
