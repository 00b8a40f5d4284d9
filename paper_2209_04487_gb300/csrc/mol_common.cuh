// Device helpers and tables shared by the molecular kernels' translation units
// (mol.cu, mol_pair.cu).  Everything here has internal linkage: each unit
// holds its own copy, and the angular tables are uploaded into every copy.
#pragma once

#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <vector>

#include "ms_internal.cuh"

namespace ms {

// Tensor maps of one species for the tiled R-space kernel: 8-byte elements
// (one complex FP32 value), boxes of TILE radial points by the rows of a
// molecule, at most 256 rows a box (a box dimension's limit): a molecule's
// rows arrive as full boxes (s, d2) and one remainder box (s_r, d2_r).
struct RspaceMaps {
  CUtensorMap s, d2;      // [n_mol * rows][nr], box TILE x min(rows, 256)
  CUtensorMap s_r, d2_r;  // same arrays, box TILE x the remainder rows (rows > 256 only)
  CUtensorMap vd, vh;     // [2 (J + 1)][nr], box TILE x 2 (J + 1)
  CUtensorMap mk;         // [1][nr], box TILE x 1
};

namespace {

__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ float2 operator+(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 operator-(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }

// ---- TMA bulk copies (cp.async.bulk) completing on an mbarrier --------------
__device__ __forceinline__ unsigned smem_u32(const void* p) {
  return (unsigned)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(unsigned long long* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}
__device__ __forceinline__ void mbar_expect_tx(unsigned long long* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, unsigned bytes, unsigned long long* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}
// 2-D tensor copy global -> shared (box of the map at element (x, y)).
__device__ __forceinline__ void tensor2d_g2s(void* dst, const CUtensorMap* map, int x, int y,
                                             unsigned long long* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
          smem_u32(dst)),
      "l"(reinterpret_cast<unsigned long long>(map)), "r"(x), "r"(y), "r"(smem_u32(bar))
      : "memory");
}
// Wait for phase `parity` of the barrier, giving up after `limit` polls.
__device__ __forceinline__ bool mbar_wait(unsigned long long* bar, unsigned parity, long long limit) {
  for (long long it = 0; it < limit; ++it) {
    unsigned done;
    asm volatile(
        "{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2; selp.u32 %0, 1, 0, p; }"
        : "=r"(done)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}
constexpr long long kWaitPolls = 1LL << 24;  // far beyond any copy's duration

__device__ __forceinline__ int j_of(int c) { return (int)sqrtf((float)c + 0.5f); }  // c = j^2+j+m


// compensated FP32 accumulation (TwoSum): hi + lo carries ~48 bits
__device__ __forceinline__ void acc2(float& hi, float& lo, float x) {
  const float t = hi + x;
  const float z = t - hi;
  lo += (hi - (t - z)) + (x - z);
  hi = t;
}

// The state's one full-magnitude rounding per step, s' = fl(s + D'), with the
// update D' = D + c s scaled by the previous step's rounding feedback c, and
// the exact residual e = (s + D') - s' of that rounding (TwoSum; the FP32
// operations must stay unfused and unreordered) folded into acc as
// Re(conj(s') e).  The rounding changed sum |s|^2 by -2 sum Re(conj(s') e) to
// first order; the next step's c = sum Re(conj(s') e) / sum |s'|^2 gives that
// back, so the norm carries one step's rounding instead of a random walk.
__device__ __forceinline__ float2 round_update(float2 sv, float2 D, float c, float& acc) {
  const float dx = fmaf(c, sv.x, D.x), dy = fmaf(c, sv.y, D.y);
  const float nx = __fadd_rn(sv.x, dx), ny = __fadd_rn(sv.y, dy);
  const float bx = __fsub_rn(nx, sv.x), by = __fsub_rn(ny, sv.y);
  const float ex = __fadd_rn(__fsub_rn(sv.x, __fsub_rn(nx, bx)), __fsub_rn(dx, bx));
  const float ey = __fadd_rn(__fsub_rn(sv.y, __fsub_rn(ny, by)), __fsub_rn(dy, by));
  acc = fmaf(nx, ex, fmaf(ny, ey, acc));
  return make_float2(nx, ny);
}

// feedback factor for the next step from the summed residual products and the
// summed |s'|^2 of a molecule (0 for an empty state)
__device__ __forceinline__ float rounding_feedback(float res, float norm2) {
  return norm2 > 0.f && isfinite(res) ? res / norm2 : 0.f;
}

// Per channel, on the two runs (j + 1, .) and (j - 1, .): .x S+ (from m - 1),
// .y Z (from m), .z S- (from m + 1), .w 0.
static __device__ float4 g_tri_up[kMaxRot], g_tri_dn[kMaxRot];

static cudaError_t upload_triplet_tables_local(const CouplEntry* dip) {
  // dipole slots: 0 Z (j-1, m), 1 Z (j+1, m), 2 S+ (j-1, m-1), 3 S+ (j+1, m-1), 4 S- (j+1, m+1), 5 S- (j-1, m+1)
  std::vector<float4> up(kMaxRot, make_float4(0.f, 0.f, 0.f, 0.f)), dn = up;
  for (int c = 0; c < kMaxRot; ++c) {
    auto cf = [&](int slot) { const CouplEntry& e = dip[c * kMaxCoupl + slot]; return e.nbr >= 0 ? e.coef : 0.f; };
    up[c] = make_float4(cf(3), cf(1), cf(4), 0.f);
    dn[c] = make_float4(cf(2), cf(0), cf(5), 0.f);
  }
  cudaError_t e = cudaMemcpyToSymbol(g_tri_up, up.data(), sizeof(float4) * kMaxRot);
  if (e != cudaSuccess) return e;
  return cudaMemcpyToSymbol(g_tri_dn, dn.data(), sizeof(float4) * kMaxRot);
}

constexpr int kTriGuard = 3;  // zero rows ahead of each term buffer


// Wait for phase `parity`, each try suspending up to hint_ns until the phase
// completes; gives up after `tries` tries (by default about 2 s in all).
__device__ __forceinline__ bool mbar_wait_sleep(unsigned long long* bar, unsigned parity, int tries = 2000,
                                                unsigned hint_ns = 1000000u) {
  for (int it = 0; it < tries; ++it) {
    unsigned done;
    asm volatile(
        "{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3; selp.u32 %0, 1, 0, p; }"
        : "=r"(done)
        : "r"(smem_u32(bar)), "r"(parity), "r"(hint_ns)
        : "memory");
    if (done) return true;
  }
  return false;
}

// persistent launch of a tiled kernel: CTA b walks molecules b, b + grid,
// ...; the grid is the plan's resident CTAs per SM (0: as many as fit) times
// the SMs, or one CTA per molecule (cps < 0)
using RspaceKernel = void (*)(SpeciesDev, MolDev, int*, const RspaceMaps);
static void launch_persistent(RspaceKernel k, int nt, int bytes, const SpeciesDev& sp, const MolDev& md, int* err,
                              const RspaceMaps& maps, cudaStream_t s) {
  cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  cudaFuncSetAttribute(k, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
  int dev = 0, nsm = 0, per = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k, nt, bytes);
  per = std::max(per, 1);
  if (sp.cps > 0) per = std::min(per, sp.cps);
  const long long fit = sp.cps < 0 ? (long long)sp.nmol : (long long)std::max(nsm, 1) * per;
  const int grid = (int)std::min<long long>(sp.nmol, fit);
  k<<<grid, nt, bytes, s>>>(sp, md, err, maps);
}


}  // namespace

// The two-points-a-thread tiled R-space pass (mol_pair.cu): the kernel of the
// species' J at tile width `tile` (and its parity-reduced form for a
// parity-reduced species), launched persistently on stream s.
void launch_rspace_pair(const SpeciesDev& sp, const MolDev& md, int* err, const RspaceMaps& maps, int tile,
                        cudaStream_t s);
// uploads the angular tables into mol_pair.cu's copy
cudaError_t upload_triplet_tables_pair(const CouplEntry* dip);
// The one-point-a-thread tiled R-space pass (mol_tile.cu) at tile width
// `tile`, launched persistently on stream s, and its copy of the tables.
void launch_rspace(const SpeciesDev& sp, const MolDev& md, int* err, const RspaceMaps& maps, int tile,
                   cudaStream_t s);
cudaError_t upload_triplet_tables_tile(const CouplEntry* dip);

}  // namespace ms
