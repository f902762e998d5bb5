// Interface step of Algorithm 1: the multiplier update
//   lambda^{n+1} = lambda^n + sigma B (2 p~^n - p~^{n-1}),
//   (B p~)_e = p_s(e) - p_t(e)   (s the upper/left tile, t the lower/right one, Section 2.4),
// on compact interface strips, plus the kernels that move strips in and out of the
// torn field.  The update is HBM-bound: 5 float reads and 1 write per interface edge.
#include "internal.cuh"

namespace ddtv {

namespace {

__device__ __forceinline__ float lam_step(float lam, float sigma, float cs, float ps, float ct, float pt) {
  // sigma * ((2 cs - ps) - (2 ct - pt)), in this order on every path
  return fmaf(sigma, fmaf(2.0f, cs, -ps) - fmaf(2.0f, ct, -pt), lam);
}

// One thread per 4 consecutive interface edges of one strip (float4 loads/stores).
// Horizontal interfaces occupy [0, nh4), vertical ones [nh4, nh4 + nv4), in units of
// float4.  Used when W and H are multiples of 4 (every strip row then starts on a
// 16-byte boundary).
__global__ void k_interface_v4(int nh4, int nv4, float sigma, const float4* __restrict__ cSB,
                               const float4* __restrict__ cST, const float4* __restrict__ pSB,
                               const float4* __restrict__ pST, float4* __restrict__ lamh,
                               const float4* __restrict__ cSR, const float4* __restrict__ cSL,
                               const float4* __restrict__ pSR, const float4* __restrict__ pSL,
                               float4* __restrict__ lamv) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < nh4 + nv4; e += gridDim.x * blockDim.x) {
    const bool h = e < nh4;
    const int q = h ? e : e - nh4;
    const float4 cs = h ? cSB[q] : cSR[q];
    const float4 ct = h ? cST[q] : cSL[q];
    const float4 ps = h ? pSB[q] : pSR[q];
    const float4 pt = h ? pST[q] : pSL[q];
    float4* lp = h ? lamh : lamv;
    float4 l = lp[q];
    l.x = lam_step(l.x, sigma, cs.x, ps.x, ct.x, pt.x);
    l.y = lam_step(l.y, sigma, cs.y, ps.y, ct.y, pt.y);
    l.z = lam_step(l.z, sigma, cs.z, ps.z, ct.z, pt.z);
    l.w = lam_step(l.w, sigma, cs.w, ps.w, ct.w, pt.w);
    lp[q] = l;
  }
}

__global__ void k_interface_v1(int nh, int nv, float sigma, const float* __restrict__ cSB,
                               const float* __restrict__ cST, const float* __restrict__ pSB,
                               const float* __restrict__ pST, float* __restrict__ lamh,
                               const float* __restrict__ cSR, const float* __restrict__ cSL,
                               const float* __restrict__ pSR, const float* __restrict__ pSL,
                               float* __restrict__ lamv) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < nh + nv; e += gridDim.x * blockDim.x) {
    if (e < nh) {
      lamh[e] = lam_step(lamh[e], sigma, cSB[e], pSB[e], cST[e], pST[e]);
    } else {
      const int q = e - nh;
      lamv[q] = lam_step(lamv[q], sigma, cSR[q], pSR[q], cSL[q], pSL[q]);
    }
  }
}

// strips <- interface values of (P1, P2): one thread per interface edge
__global__ void k_extract(Grid g, const float* __restrict__ P1, const float* __restrict__ P2, Strips s) {
  const int nh = (g.NR - 1) * g.W, nv = (g.NC - 1) * g.H;
  const int W2 = g.W + g.NC;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < nh + nv; e += gridDim.x * blockDim.x) {
    if (e < nh) {
      const int a = e / g.W, j = e % g.W;
      const int rs = part_start(a + 1, g.H, g.NR) + a;  // bottom side of tile row a
      s.SB[e] = P1[(size_t)rs * g.W + j];
      s.ST[e] = P1[(size_t)(rs + 1) * g.W + j];
    } else {
      const int q = e - nh, b = q / g.H, i = q % g.H;
      const int cs = part_start(b + 1, g.W, g.NC) + b;  // right side of tile column b
      s.SR[q] = P2[(size_t)i * W2 + cs];
      s.SL[q] = P2[(size_t)i * W2 + cs + 1];
    }
  }
}

__global__ void k_scatter(Grid g, Strips s, float* __restrict__ P1, float* __restrict__ P2) {
  const int nh = (g.NR - 1) * g.W, nv = (g.NC - 1) * g.H;
  const int W2 = g.W + g.NC;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < nh + nv; e += gridDim.x * blockDim.x) {
    if (e < nh) {
      const int a = e / g.W, j = e % g.W;
      const int rs = part_start(a + 1, g.H, g.NR) + a;
      P1[(size_t)rs * g.W + j] = s.SB[e];
      P1[(size_t)(rs + 1) * g.W + j] = s.ST[e];
    } else {
      const int q = e - nh, b = q / g.H, i = q % g.H;
      const int cs = part_start(b + 1, g.W, g.NC) + b;
      P2[(size_t)i * W2 + cs] = s.SR[q];
      P2[(size_t)i * W2 + cs + 1] = s.SL[q];
    }
  }
}

// Batched multiplier update over every image of a batch (W, H multiples of 4): the
// float4 elements of all images are numbered consecutively, image by image.
__global__ void k_interface_batch(BatchIfaceArgs B, int total4) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < total4; e += gridDim.x * blockDim.x) {
    int lo = 0, hi = B.n_img;  // find the image: elem_base[img] <= e < elem_base[img + 1]
    while (hi - lo > 1) {
      const int mid = (lo + hi) >> 1;
      if (B.elem_base[mid] <= e) lo = mid; else hi = mid;
    }
    const int img = lo;
    const LocalArgs& A = B.args[img];
    const Strips cur = B.strips[2 * img + B.cur_set], prev = B.strips[2 * img + 1 - B.cur_set];
    const float sigma = B.sigma[img];
    const int q = e - B.elem_base[img];
    const int nh4 = (A.g.NR - 1) * A.g.W / 4;
    const bool h = q < nh4;
    const int qq = h ? q : q - nh4;
    const float4 cs = h ? reinterpret_cast<const float4*>(cur.SB)[qq] : reinterpret_cast<const float4*>(cur.SR)[qq];
    const float4 ct = h ? reinterpret_cast<const float4*>(cur.ST)[qq] : reinterpret_cast<const float4*>(cur.SL)[qq];
    const float4 ps = h ? reinterpret_cast<const float4*>(prev.SB)[qq] : reinterpret_cast<const float4*>(prev.SR)[qq];
    const float4 pt = h ? reinterpret_cast<const float4*>(prev.ST)[qq] : reinterpret_cast<const float4*>(prev.SL)[qq];
    float4* lp = reinterpret_cast<float4*>(const_cast<float*>(h ? A.lamh : A.lamv));
    float4 l = lp[qq];
    l.x = lam_step(l.x, sigma, cs.x, ps.x, ct.x, pt.x);
    l.y = lam_step(l.y, sigma, cs.y, ps.y, ct.y, pt.y);
    l.z = lam_step(l.z, sigma, cs.z, ps.z, ct.z, pt.z);
    l.w = lam_step(l.w, sigma, cs.w, ps.w, ct.w, pt.w);
    lp[qq] = l;
  }
}

int grid_for(long long n, int block) {
  long long b = (n + block - 1) / block;
  if (b < 1) b = 1;
  if (b > 152 * 16) b = 152 * 16;  // grid-stride beyond 16 blocks per SM
  return (int)b;
}

}  // namespace

cudaError_t launch_interface(const Grid& g, float sigma, Strips cur, Strips prev, float* lamh, float* lamv,
                             cudaStream_t st) {
  const int nh = (g.NR - 1) * g.W, nv = (g.NC - 1) * g.H;
  if (nh + nv == 0) return cudaSuccess;
  const int block = 256;
  if (g.W % 4 == 0 && g.H % 4 == 0) {
    const int nh4 = nh / 4, nv4 = nv / 4;
    k_interface_v4<<<grid_for(nh4 + nv4, block), block, 0, st>>>(
        nh4, nv4, sigma, (const float4*)cur.SB, (const float4*)cur.ST, (const float4*)prev.SB,
        (const float4*)prev.ST, (float4*)lamh, (const float4*)cur.SR, (const float4*)cur.SL, (const float4*)prev.SR,
        (const float4*)prev.SL, (float4*)lamv);
  } else {
    k_interface_v1<<<grid_for(nh + nv, block), block, 0, st>>>(nh, nv, sigma, cur.SB, cur.ST, prev.SB, prev.ST,
                                                                lamh, cur.SR, cur.SL, prev.SR, prev.SL, lamv);
  }
  return cudaGetLastError();
}

cudaError_t launch_interface_batch(const BatchIfaceArgs& a, int total4, cudaStream_t st) {
  if (total4 == 0) return cudaSuccess;
  k_interface_batch<<<grid_for(total4, 256), 256, 0, st>>>(a, total4);
  return cudaGetLastError();
}

cudaError_t launch_extract_strips(const Grid& g, const float* P1, const float* P2, Strips s, cudaStream_t st) {
  const int n = (g.NR - 1) * g.W + (g.NC - 1) * g.H;
  if (n == 0) return cudaSuccess;
  k_extract<<<grid_for(n, 256), 256, 0, st>>>(g, P1, P2, s);
  return cudaGetLastError();
}

cudaError_t launch_scatter_strips(const Grid& g, Strips s, float* P1, float* P2, cudaStream_t st) {
  const int n = (g.NR - 1) * g.W + (g.NC - 1) * g.H;
  if (n == 0) return cudaSuccess;
  k_scatter<<<grid_for(n, 256), 256, 0, st>>>(g, s, P1, P2);
  return cudaGetLastError();
}

}  // namespace ddtv
