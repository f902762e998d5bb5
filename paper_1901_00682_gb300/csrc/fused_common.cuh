// Device helpers shared by the fused kernels: shared-memory and cluster addressing,
// DSMEM stores, the split cluster barrier, packed float32 pairs, bounded mbarrier
// waits, asynchronous copies, and the shared-memory layouts of the 128 x 128 kernels.
#pragma once

#include "internal.cuh"

namespace ddtv {
namespace {

__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint32_t map_rank(uint32_t addr, int rank) {
  uint32_t out;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(out) : "r"(addr), "r"(rank));
  return out;
}

__device__ __forceinline__ void st_cluster(uint32_t addr, float v) {
  asm volatile("st.shared::cluster.f32 [%0], %1;" ::"r"(addr), "f"(v) : "memory");
}

__device__ __forceinline__ void st_cluster_f64(uint32_t addr, double v) {
  asm volatile("st.shared::cluster.f64 [%0], %1;" ::"r"(addr), "d"(v) : "memory");
}

// Packed float32 pairs (sm_100+ `*.f32x2`): one instruction performs the operation on
// two lanes, each rounded exactly as the scalar instruction, so packed and scalar code
// give identical bits.
typedef unsigned long long f32x2;

__device__ __forceinline__ f32x2 pk2(float lo, float hi) {
  f32x2 r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
  return r;
}
__device__ __forceinline__ float lo2(f32x2 v) {
  float a;
  asm("mov.b64 {%0, _}, %1;" : "=f"(a) : "l"(v));
  return a;
}
__device__ __forceinline__ float hi2(f32x2 v) {
  float b;
  asm("mov.b64 {_, %0}, %1;" : "=f"(b) : "l"(v));
  return b;
}
__device__ __forceinline__ f32x2 add2(f32x2 a, f32x2 b) {
  f32x2 r;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
  return r;
}
__device__ __forceinline__ f32x2 sub2(f32x2 a, f32x2 b) {
  f32x2 r;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
  return r;
}
__device__ __forceinline__ f32x2 mul2(f32x2 a, f32x2 b) {
  f32x2 r;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
  return r;
}
// a * b + c, one rounding per lane (fmaf)
__device__ __forceinline__ f32x2 fma2(f32x2 a, f32x2 b, f32x2 c) {
  f32x2 r;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(a), "l"(b), "l"(c));
  return r;
}

template <bool RELEASE>
__device__ __forceinline__ void cluster_arrive() {
  if (RELEASE)
    asm volatile("barrier.cluster.arrive.release.aligned;" ::: "memory");
  else
    asm volatile("barrier.cluster.arrive.relaxed.aligned;" ::: "memory");
}

__device__ __forceinline__ void cluster_wait() { asm volatile("barrier.cluster.wait.acquire.aligned;" ::: "memory"); }

// p_update with the clamp to [-lim, lim]; lim = 0 pins an inactive dof at 0
__device__ __forceinline__ void p_update_lim(float& p, float& pbar, float du, float phat, const Coef& c, float lim) {
  const float t = p_target(p, du, phat, c);
  const float pn = clamp_abs(t, lim);
  pbar = fmaf(c.th, pn - p, pn);
  p = pn;
}

// ---------------------------------------------------------------------------
// Full-tile kernel: every subdomain is exactly 128 x 128 (the partition of the
// benchmark workloads).  Same arithmetic as k_fused, without any per-pixel
// boundary test: the band's halo rows live in the shared arrays (row 0 of sU is
// the row above the band, row TR of sQ1 the row below it), the tile's bottom side
// is the "row below" of the last CTA, and the right side's dofs are updated by
// lanes 0..R-1 of each thread row's first warp (one dof per lane).
template <int R, int TR>
struct FullLayout {
  static constexpr int BW = 128;
  static constexpr int BAND = TR * R;
  static constexpr int US = BW + 1;                    // u row stride; index 0 = zero pad
  static constexpr int QS = BW + 1;                    // pbar2 row stride; index 128 = right side
  static constexpr int U = 0;                          // (BAND + 1) x US: row 0 = row above the band
  static constexpr int Q2 = U + (BAND + 1) * US;       // BAND x QS
  static constexpr int Q1 = Q2 + BAND * QS;            // (TR + 1) x BW: first-row pbar1 per thread row; row TR = below
  static constexpr int F = Q1 + (TR + 1) * BW;         // BAND x BW
  static constexpr int PR = F + BAND * BW;             // BAND right-side p
  static constexpr int HR = PR + BAND;                 // BAND right-side phat
  static constexpr int CO = (HR + BAND + 3) & ~3;      // kMaxSmemCoef x 8 coefficients (16-byte aligned)
  static constexpr int FLOATS = CO + 8 * 64;
  static constexpr size_t BYTES = sizeof(float) * FLOATS;
  static constexpr int kMaxSmemCoef = 64;
};

constexpr unsigned kWaitLimit = 1000;
constexpr unsigned kSuspendHintNs = 1000000;

__device__ __forceinline__ void mbar_init(uint32_t addr, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(addr), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive_local(uint32_t addr) {
  asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.release.cta.shared::cta.b64 st, [%0];\n\t}" ::"r"(addr)
               : "memory");
}

__device__ __forceinline__ void mbar_arrive_remote(uint32_t cluster_addr) {
  asm volatile("mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0];" ::"r"(cluster_addr) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t addr, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2, %3;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(addr), "r"(parity), "r"(kSuspendHintNs)
      : "memory");
  return ok != 0;
}

// bounded wait; returns false (and the caller records the timeout) when the limit runs out
__device__ __forceinline__ bool mbar_wait(uint32_t addr, uint32_t parity) {
  for (unsigned it = 0; it < kWaitLimit; ++it)
    if (mbar_try_wait(addr, parity)) return true;
  return false;
}

__device__ __forceinline__ void st_cluster_v4(uint32_t addr, float4 v) {
  asm volatile("st.shared::cluster.v4.f32 [%0], {%1, %2, %3, %4};" ::"r"(addr), "f"(v.x), "f"(v.y), "f"(v.z),
               "f"(v.w)
               : "memory");
}

__device__ __forceinline__ void st_async_f32(uint32_t remote_addr, float v, uint32_t remote_mbar) {
  asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.b32 [%0], %1, [%2];" ::"r"(remote_addr),
               "r"(__float_as_uint(v)), "r"(remote_mbar)
               : "memory");
}

// two floats into a neighbour CTA's shared memory (8-byte aligned), counted on its mbarrier
__device__ __forceinline__ void st_async_v2(uint32_t remote_addr, float a, float b, uint32_t remote_mbar) {
  asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.v2.b32 [%0], {%1, %2}, [%3];" ::"r"(remote_addr),
               "r"(__float_as_uint(a)), "r"(__float_as_uint(b)), "r"(remote_mbar)
               : "memory");
}

// four floats into a neighbour CTA's shared memory (16-byte aligned), counted on its mbarrier
__device__ __forceinline__ void st_async_v4_f32(uint32_t remote_addr, float a, float b, float c, float d,
                                                uint32_t remote_mbar) {
  asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.v4.b32 [%0], {%1, %2, %3, %4}, [%5];" ::"r"(
                   remote_addr),
               "r"(__float_as_uint(a)), "r"(__float_as_uint(b)), "r"(__float_as_uint(c)), "r"(__float_as_uint(d)),
               "r"(remote_mbar)
               : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint32_t addr, uint32_t bytes) {
  asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.expect_tx.release.cta.shared::cta.b64 st, [%0], %1;\n\t}" ::"r"(addr),
               "r"(bytes)
               : "memory");
}

__device__ __forceinline__ void cp_async4(float* dst_smem, const float* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(smem_addr(dst_smem)), "l"(src) : "memory");
}
// 16-byte copy (both addresses 16-byte aligned), cached in L2 only
__device__ __forceinline__ void cp_async16(float* dst_smem, const float* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_addr(dst_smem)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

// Source of the subdomains a persistent batch kernel iterates over: the number of
// subdomains, their image's arguments and grid position, the strips that receive
// their interface values, and a call of the tile body with the image's fidelity as a
// compile-time constant (FidC).
template <int V>
struct FidC {
  static constexpr int value = V;
};

// The batch's work list: (image, tile) with the fidelity, parameters and coefficients
// of each image.
struct BatchTiles {
  const BatchArgs& B;
  int total;
  static constexpr bool kBatch = true;
  __device__ int count() const { return total; }
  __device__ int inner() const { return B.args[0].K; }
  __device__ int image(int t) const { return B.tile_img[t]; }
  __device__ const LocalArgs& args(int t) const { return B.args[B.tile_img[t]]; }
  __device__ int local(int t) const { return t - B.tile_base[B.tile_img[t]]; }
  __device__ int fid(int t) const { return B.fid[B.tile_img[t]]; }
  __device__ Strips out(int t) const { return B.strips[2 * B.tile_img[t] + B.write_set]; }
  __device__ int* err() const { return B.args[0].err; }
  template <class Body>
  __device__ void dispatch(int t, Body&& body) const {
    switch (fid(t)) {
      case FID_L2: body(FidC<FID_L2>{}); break;
      case FID_L1: body(FidC<FID_L1>{}); break;
      default: body(FidC<FID_SEG>{}); break;
    }
  }
};

}  // namespace
}  // namespace ddtv
