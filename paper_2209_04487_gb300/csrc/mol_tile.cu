// Tiled R-space pass with one radial point a thread (MS_KERN_TILE): the
// kernels and their launch.  The pass is the R-space half of the
// split-operator step of Eqs. 4-7 (the potential phases of Eqs. 6-7, the
// exponential of the field interaction, the absorbing mask) and the
// populations and molecular dipole it reports.  A translation unit of its
// own, so that it compiles beside mol.cu.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <cstddef>
#include <type_traits>

#include "mol_common.cuh"

namespace ms {
namespace {

// One row of the tiled kernel's row table (built per molecule).
struct RowT {
  float4 cu, cd;  // theta x coupling on the runs (j + 1, .) and (j - 1, .)
  float4 du, dd;  // dipole coefficients on the runs
  float2 ph;      // e^{i m phi_E}
  int ou, od;     // byte offsets of the two runs in a term buffer (from its base)
  int vo, pad;    // byte offset of the row's (surface, j) potential row in a table tile
};

// Layout of the tiled R-space kernel for basis size J and tile width TILE
// (32, 16 or 8 radial points).  A warp covers RPL = 32 / TILE rows of one tile
// (lane = part * TILE + point, part = lane / TILE) and NW warps of RPW row
// slots each cover the 2 (J + 1)^2 rows: warp w owns rows RPL (w + NW i) +
// part.  Up to J = 8 (tiles of 32 or 16) RPW = J + 1 and the rows split
// exactly, so every row index, buffer offset and stride is known at compile
// time.  From J = 9 on (tiles of 8, 578 rows at J = 16) RPW = 6 and the last
// slots run past the rows: those padded rows stay zero, their row-table
// entries point at the zero guard rows, and they are neither summed nor
// written.  A row of a tile is SEG = 8 TILE bytes; the RPL rows of a slot
// are contiguous, so a warp's 32 lanes always read 256 contiguous bytes.
// Shared memory, from a 128-byte aligned base:
//   [2 RP] s and d2 of the tile, [2][NV] e^{-iV dtau} - 1, [2][NV]
//   e^{-iV dtau/2} (double buffered), [1] mask, two term buffers of
//   kTriGuard + RP rows, the row table of the molecule (RP = padded rows).
// With 16-point tiles the J = 8 kernel needs 109 KB, so two CTAs share an SM
// and one's barriers and copies overlap the other's arithmetic; the J = 16
// kernel needs 211 KB at 800 threads.
template <int J, int TILE>
struct RsDims {
  static constexpr int NROT = (J + 1) * (J + 1), ROWS = 2 * NROT, NV = 2 * (J + 1);
  static constexpr int RPL = 32 / TILE;
  static constexpr int RPW = TILE == 8 ? 6 : J + 1;
  static constexpr int NW = ((ROWS + RPL - 1) / RPL + RPW - 1) / RPW, NT = 32 * NW;
  static constexpr int RP = NW * RPW * RPL;  // rows with padding
  static constexpr bool EXACT = RP == ROWS;
  static constexpr int SEG = TILE * (int)sizeof(float2);
  static constexpr int BOXR = ROWS < 256 ? ROWS : 256, NBOX = (ROWS + BOXR - 1) / BOXR;
  static constexpr int LASTR = ROWS - (NBOX - 1) * BOXR;  // rows of the last box
  static constexpr int TBB = (kTriGuard + RP) * SEG;      // bytes of a term buffer
  static constexpr int O_STG = 0, O_VD = O_STG + 2 * RP * SEG, O_VH = O_VD + 2 * NV * SEG;
  static constexpr int O_MK = O_VH + 2 * NV * SEG, O_TB = O_MK + (SEG < 128 ? 128 : SEG), O_RT = O_TB + 2 * TBB;
  static constexpr int BYTES = 128 + O_RT + RP * (int)sizeof(RowT);
  static constexpr int MINB = TILE == 16 ? 2 : (J <= 4 ? 3 : 1);
  static_assert(TILE == 8 || TILE == 16 || TILE == 32, "tile of 8, 16 or 32 radial points");
  static_assert(TILE == 8 || 2 * (J + 1) % RPL == 0, "rows split evenly over the warps");
  static_assert(NT <= 1024 && BYTES <= 227 * 1024, "one CTA per molecule fits");
  static_assert((RP * SEG) % 128 == 0 && (NV * SEG) % 128 == 0 && (BOXR * SEG) % 128 == 0,
                "tensor-copy destinations 128-byte aligned");
};

template <int OFF>
__device__ __forceinline__ float2 lds2(const unsigned char* base, int off) {
  return *reinterpret_cast<const float2*>(base + off + OFF);
}
template <int OFF>
__device__ __forceinline__ void sts2(unsigned char* base, int off, float2 v) {
  *reinterpret_cast<float2*>(base + off + OFF) = v;
}

// Persistent: CTA b runs molecules b, b + gridDim.x, ...; the first tile of
// its next molecule is requested as soon as the last tile of the current one
// has left the staging buffer.  The molecule's frame field and term count
// come from its record (mol_field_kernel).
template <int J, int TILE>
__global__ void __launch_bounds__(RsDims<J, TILE>::NT, RsDims<J, TILE>::MINB)
    mol_rspace_kernel(SpeciesDev sp, MolDev md, int* err, const __grid_constant__ RspaceMaps maps) {
  using D = RsDims<J, TILE>;
  constexpr int NROT = D::NROT, ROWS = D::ROWS, NV = D::NV, NW = D::NW, RPW = D::RPW, NT = D::NT;
  constexpr int RPL = D::RPL, SEG = D::SEG, TBB = D::TBB, G0 = kTriGuard * SEG;
  constexpr int SLOT = RPL * SEG;                 // bytes of one warp's rows in a tile buffer
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ __align__(8) unsigned long long s_bar[1];
  __shared__ float s_rot[9];
  __shared__ double s_mu[3], s_abs[2];
  __shared__ float2 s_ph[2 * kMaxJ + 1];
  __shared__ float s_red[NW][10];
  __shared__ float s_fin[8], s_fin_lo[2];

  const int NR = sp.nr;
  const int t = threadIdx.x, lane = t & 31, w = t >> 5;
  const int half = lane / TILE, pt = lane % TILE;
  const int pad = (int)((128u - (smem_u32(smem_raw) & 127u)) & 127u);
  unsigned char* const sm = smem_raw;
  // this thread's byte offsets: own rows RPL (w + NW i) + half at point pt, and their row-table entries
  const int own = pad + w * SLOT + lane * 8;
  const int rtw = pad + D::O_RT + (RPL * w + half) * (int)sizeof(RowT);
  auto issue = [&](int mol, int ck) {
    const int r0 = ck * TILE, b = ck & 1;
    unsigned char* base = sm + pad;
#pragma unroll
    for (int k = 0; k < D::NBOX; ++k) {  // the molecule's rows, in boxes of at most 256
      const bool last = k == D::NBOX - 1 && D::NBOX > 1;
      tensor2d_g2s(base + D::O_STG + k * D::BOXR * SEG, last ? &maps.s_r : &maps.s, r0, mol * ROWS + k * D::BOXR,
                   &s_bar[0]);
      tensor2d_g2s(base + D::O_STG + (D::RP + k * D::BOXR) * SEG, last ? &maps.d2_r : &maps.d2, r0,
                   mol * ROWS + k * D::BOXR, &s_bar[0]);
    }
    tensor2d_g2s(base + D::O_VD + b * NV * SEG, &maps.vd, r0, 0, &s_bar[0]);
    tensor2d_g2s(base + D::O_VH + b * NV * SEG, &maps.vh, r0, 0, &s_bar[0]);
    tensor2d_g2s(base + D::O_MK, &maps.mk, r0, 0, &s_bar[0]);
  };
  constexpr unsigned kChunkBytes = (2 * ROWS + 2 * NV + 1) * SEG;  // what the copies of one tile deliver
  const int nchunks = NR / TILE;  // even: NR is 64, 128 or 256

  int lm = blockIdx.x;
  if (t == 0) {
    mbar_init(&s_bar[0], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    mbar_expect_tx(&s_bar[0], kChunkBytes);
    issue(lm, 0);
  }
  for (int q = t; q < kTriGuard * TILE; q += NT) {
    reinterpret_cast<float2*>(sm + pad + D::O_TB)[q] = make_float2(0.f, 0.f);
    reinterpret_cast<float2*>(sm + pad + D::O_TB + TBB)[q] = make_float2(0.f, 0.f);
  }
  if constexpr (!D::EXACT) {  // padded staging rows: zero, and never written by the copies
    for (int q = t; q < (D::RP - ROWS) * TILE; q += NT) {
      reinterpret_cast<float2*>(sm + pad + D::O_STG + ROWS * SEG)[q] = make_float2(0.f, 0.f);
      reinterpret_cast<float2*>(sm + pad + D::O_STG + (D::RP + ROWS) * SEG)[q] = make_float2(0.f, 0.f);
    }
  }
  // ground rows: q = RPL (w + NW i) + part < NROT; rows past ROWS are padding
  auto ground = [&](int i) { return RPL * (w + NW * i) + half < NROT; };
  auto valid = [&](int i) { return D::EXACT || RPL * (w + NW * i) + half < ROWS; };

  for (; lm < sp.nmol; lm += gridDim.x) {
    const int m = sp.mol[lm];
    __syncthreads();  // the previous molecule's outputs are written: its records may be replaced
    const float4 f = __ldg(&sp.fld[lm]);  // (theta E'_z, theta E'_x/2, theta E'_y/2, terms)
    const int nterms = __float_as_int(f.w);
    if (t <= J) {  // e^{i t phi_E} by binary powers of e^{i phi_E} = (E'_x + i E'_y)/E_perp
      const float ep = sqrtf(f.y * f.y + f.z * f.z);
      float2 e1 = ep > 0.f ? make_float2(f.y / ep, f.z / ep) : make_float2(1.f, 0.f);
      float2 pw = make_float2(1.f, 0.f);
      for (int k = t; k > 0; k >>= 1) {
        if (k & 1) pw = cmul(pw, e1);
        e1 = cmul(e1, e1);
      }
      s_ph[J + t] = pw;
      s_ph[J - t] = make_float2(pw.x, -pw.y);
    }
    for (int q = t; q < 14; q += NT) {  // rotation, previous dipole, absorbed norm so far
      if (q < 9) s_rot[q] = md.rot[9 * (long long)m + q];
      else if (q < 12) s_mu[q - 9] = md.mu[3 * (long long)m + (q - 9)];
      else s_abs[q - 12] = md.absorbed[2 * (long long)m + (q - 12)];
    }
    const float cfix = md.ncorr[m];  // rounding feedback of the previous step
    __syncthreads();
    for (int q = t; q < D::RP; q += NT) {  // the row table of this molecule (padding: zero, guard rows)
      if (!D::EXACT && q >= ROWS) {
        RowT r;
        r.cu = r.cd = r.du = r.dd = make_float4(0.f, 0.f, 0.f, 0.f);
        r.ph = make_float2(1.f, 0.f);
        r.ou = r.od = D::O_TB;
        r.vo = 0;
        r.pad = 0;
        *reinterpret_cast<RowT*>(sm + pad + D::O_RT + q * (int)sizeof(RowT)) = r;
        continue;
      }
      // theta E_perp / 2 on the X runs and theta E'_z on the Z runs (frame turned so E'_y = 0)
      const float ep = sqrtf(f.y * f.y + f.z * f.z), ez = f.x;
      const int sf = q >= NROT, c = q - sf * NROT, j = j_of(c), mm = c - j * j - j;
      const int other = kTriGuard + (1 - sf) * NROT;
      RowT r;
      r.ph = s_ph[mm + J];
      const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
      r.du = j < J ? g_tri_up[c] : z4;
      r.dd = j > 0 ? g_tri_dn[c] : z4;
      r.cu = make_float4(ep * r.du.x, ez * r.du.y, ep * r.du.z, 0.f);
      r.cd = make_float4(ep * r.dd.x, ez * r.dd.y, ep * r.dd.z, 0.f);
      r.ou = D::O_TB + (j < J ? (other + c + 2 * j + 1) * SEG : 0);
      r.od = D::O_TB + (j > 0 ? (other + c - 2 * j - 1) * SEG : 0);
      r.vo = (sf * (J + 1) + j) * SEG;
      r.pad = 0;
      *reinterpret_cast<RowT*>(sm + pad + D::O_RT + q * (int)sizeof(RowT)) = r;
    }
    float2 sv[RPW], dv[RPW], sacc[RPW];
    float p_hi[2] = {0.f, 0.f}, p_lo[2] = {0.f, 0.f};  // populations, compensated
    float a_gf = 0.f, a_ef = 0.f, dP = 0.f, dQ = 0.f, dZ = 0.f, rnd = 0.f;
    float2* gs = sp.psi + (long long)lm * ROWS * NR;

    // one coupling-series term reading term buffer P (compile-time), writing
    // the other one unless it is the last
    auto term = [&](auto Pc, int n) {
      constexpr int P = decltype(Pc)::value;
      const float cn = 1.f / (float)n;
      const bool store = n < nterms;
#pragma unroll
      for (int i = 0; i < RPW; ++i) {
        const unsigned char* rt = sm + rtw + NW * RPL * i * (int)sizeof(RowT);
        const float4 cu = *reinterpret_cast<const float4*>(rt + offsetof(RowT, cu));
        const float4 cd = *reinterpret_cast<const float4*>(rt + offsetof(RowT, cd));
        const int2 oo = *reinterpret_cast<const int2*>(rt + offsetof(RowT, ou));
        const int ou = pad + pt * 8 + oo.x, od = pad + pt * 8 + oo.y;
        const float2 u0 = lds2<P * TBB>(sm, ou), u1 = lds2<P * TBB + SEG>(sm, ou),
                     u2 = lds2<P * TBB + 2 * SEG>(sm, ou);
        const float2 d0 = lds2<P * TBB>(sm, od), d1 = lds2<P * TBB + SEG>(sm, od),
                     d2 = lds2<P * TBB + 2 * SEG>(sm, od);
        float ax = cu.x * u0.x, ay = cu.x * u0.y;
        ax = fmaf(cu.y, u1.x, ax); ay = fmaf(cu.y, u1.y, ay);
        ax = fmaf(cu.z, u2.x, ax); ay = fmaf(cu.z, u2.y, ay);
        ax = fmaf(cd.x, d0.x, ax); ay = fmaf(cd.x, d0.y, ay);
        ax = fmaf(cd.y, d1.x, ax); ay = fmaf(cd.y, d1.y, ay);
        ax = fmaf(cd.z, d2.x, ax); ay = fmaf(cd.z, d2.y, ay);
        const float2 o = make_float2(-cn * ay, cn * ax);  // i (theta/n) M in
        sacc[i].x += o.x;
        sacc[i].y += o.y;
        if (store) sts2<(1 - P) * TBB + G0>(sm, own + D::O_TB + NW * i * SLOT, o);
      }
      if (store) __syncthreads();
    };

    // one tile with the buffer parity B known at compile time; false on a timeout
    auto chunk = [&](auto Bc, int ck) -> bool {
      constexpr int B = decltype(Bc)::value;
      constexpr int OVD = D::O_VD + B * NV * SEG, OVH = D::O_VH + B * NV * SEG;
      const bool ok = mbar_wait_sleep(&s_bar[0], (unsigned)B);
      if (!__syncthreads_and(ok)) {
        if (t == 0) atomicOr(err, kErrTimeout);
        if (!ok) mbar_wait_sleep(&s_bar[0], (unsigned)B);
        return false;
      }
      const float mk = reinterpret_cast<const float2*>(sm + pad + D::O_MK)[pt].x;
      // ---- s, d2; eta = e^{i m phi} V^{1/2} u into term buffer 0
#pragma unroll
      for (int i = 0; i < RPW; ++i) {
        sv[i] = lds2<D::O_STG>(sm, own + NW * i * SLOT);
        dv[i] = lds2<D::O_STG + D::RP * SEG>(sm, own + NW * i * SLOT);
        sacc[i] = make_float2(0.f, 0.f);
        if (nterms > 0) {
          const unsigned char* rt = sm + rtw + NW * RPL * i * (int)sizeof(RowT);
          const int vo = pad + pt * 8 + *reinterpret_cast<const int*>(rt + offsetof(RowT, vo));
          const float2 vh = lds2<OVH>(sm, vo);
          const float2 ph = *reinterpret_cast<const float2*>(rt + offsetof(RowT, ph));
          sts2<D::O_TB + G0>(sm, own + NW * i * SLOT, cmul(ph, cmul(vh, sv[i] + dv[i])));
        }
      }
      __syncthreads();
      if (t == 0) {  // the staging buffer is free: the next tile, or the next molecule's first
        if (ck + 1 < nchunks) {
          mbar_expect_tx(&s_bar[0], kChunkBytes);
          issue(lm, ck + 1);
        } else if (lm + (int)gridDim.x < sp.nmol) {
          mbar_expect_tx(&s_bar[0], kChunkBytes);
          issue(lm + (int)gridDim.x, 0);
        }
      }
      for (int n = 1; n <= nterms; n += 2) {
        term(std::integral_constant<int, 0>(), n);
        if (n + 1 <= nterms) term(std::integral_constant<int, 1>(), n + 1);
      }
      // ---- d1 = (V - 1) u + V^{1/2} e^{-i m phi} S ; mask ; s' = s + (d2 + d1) + cfix s
      const int sbo = (nterms & 1) * TBB;  // s' buffer: not read by the last term
      float2* gsw = gs + (long long)(RPL * w + half) * NR + ck * TILE + pt;
#pragma unroll
      for (int i = 0; i < RPW; ++i) {
        const unsigned char* rt = sm + rtw + NW * RPL * i * (int)sizeof(RowT);
        const int vo = pad + pt * 8 + *reinterpret_cast<const int*>(rt + offsetof(RowT, vo));
        const float2 u = sv[i] + dv[i];
        const float2 vd = lds2<OVD>(sm, vo);
        float2 d1 = cmul(vd, u);
        if (nterms > 0) {
          const float2 vh = lds2<OVH>(sm, vo);
          const float2 ph = *reinterpret_cast<const float2*>(rt + offsetof(RowT, ph));
          d1 = d1 + cmul(vh, cmul(make_float2(ph.x, -ph.y), sacc[i]));
        }
        const bool gr = ground(i);
        if (mk < 1.f) {
          const float px = u.x + d1.x, py = u.y + d1.y;
          d1.x = fmaf(mk - 1.f, u.x, mk * d1.x);
          d1.y = fmaf(mk - 1.f, u.y, mk * d1.y);
          const float dd = (1.f - mk * mk) * fmaf(px, px, py * py);
          if (gr) a_gf += dd; else a_ef += dd;
        }
        const float2 sn = round_update(sv[i], dv[i] + d1, cfix, rnd);
        if (valid(i)) gsw[(long long)(RPL * NW * i) * NR] = sn;  // padded rows: zero, not stored
        sts2<D::O_TB + G0>(sm, own + sbo + NW * i * SLOT, sn);
        sv[i] = sn;
        const float b2 = fmaf(sn.x, sn.x, sn.y * sn.y);
        if (gr) acc2(p_hi[0], p_lo[0], b2);  // compensated from the first term on
        else acc2(p_hi[1], p_lo[1], b2);
      }
      __syncthreads();
      // ---- dipole in the molecule frame: sum_c conj(g_c) (A e)_c for A = Z, S+, S-
      float2 accP = make_float2(0.f, 0.f), accM = accP, accZ = accP;
#pragma unroll
      for (int i = 0; i < RPW; ++i) {
        if (ground(i)) {
          const unsigned char* rt = sm + rtw + NW * RPL * i * (int)sizeof(RowT);
          const float2 gc = sv[i];
          const float4 du = *reinterpret_cast<const float4*>(rt + offsetof(RowT, du));
          const float4 dd = *reinterpret_cast<const float4*>(rt + offsetof(RowT, dd));
          const int2 oo = *reinterpret_cast<const int2*>(rt + offsetof(RowT, ou));
          const int a = pad + pt * 8 + oo.x + sbo, c = pad + pt * 8 + oo.y + sbo;
          const float2 u0 = lds2<0>(sm, a), u1 = lds2<SEG>(sm, a), u2 = lds2<2 * SEG>(sm, a);
          const float2 e0 = lds2<0>(sm, c), e1 = lds2<SEG>(sm, c), e2 = lds2<2 * SEG>(sm, c);
          const float2 wP = make_float2(fmaf(du.x, u0.x, dd.x * e0.x), fmaf(du.x, u0.y, dd.x * e0.y));
          const float2 wZ = make_float2(fmaf(du.y, u1.x, dd.y * e1.x), fmaf(du.y, u1.y, dd.y * e1.y));
          const float2 wM = make_float2(fmaf(du.z, u2.x, dd.z * e2.x), fmaf(du.z, u2.y, dd.z * e2.y));
          accZ.x += fmaf(gc.x, wZ.x, gc.y * wZ.y);
          accZ.y += fmaf(gc.x, wZ.y, -gc.y * wZ.x);
          accP.x += fmaf(gc.x, wP.x, gc.y * wP.y);
          accP.y += fmaf(gc.x, wP.y, -gc.y * wP.x);
          accM.x += fmaf(gc.x, wM.x, gc.y * wM.y);
          accM.y += fmaf(gc.x, wM.y, -gc.y * wM.x);
        }
      }
      dP += accP.x + accM.x;
      dQ += accP.y - accM.y;
      dZ += 2.f * accZ.x;
      return true;
    };

    for (int ck = 0; ck < nchunks; ck += 2) {
      if (!chunk(std::integral_constant<int, 0>(), ck)) return;
      if (!chunk(std::integral_constant<int, 1>(), ck + 1)) return;
    }
    // ---- block reduction: populations compensated, the rest plain FP32
    {
      float v[8] = {p_hi[0], p_hi[1], a_gf, a_ef, dP, dQ, dZ, rnd};
      float lo[2] = {p_lo[0], p_lo[1]};
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
        for (int k = 0; k < 2; ++k) {
          const float h2 = __shfl_xor_sync(0xffffffffu, v[k], o);
          const float l2 = __shfl_xor_sync(0xffffffffu, lo[k], o);
          acc2(v[k], lo[k], h2);
          lo[k] += l2;
        }
#pragma unroll
        for (int k = 2; k < 8; ++k) v[k] += __shfl_xor_sync(0xffffffffu, v[k], o);
      }
      if (lane == 0) {
#pragma unroll
        for (int k = 0; k < 7; ++k) s_red[w][k] = v[k];
        s_red[w][7] = lo[0];
        s_red[w][8] = lo[1];
        s_red[w][9] = v[7];
      }
      __syncthreads();
      if (t < 8) {
        float hi = 0.f, l = 0.f;
        for (int ww = 0; ww < NW; ++ww) {
          acc2(hi, l, s_red[ww][t < 7 ? t : 9]);
          if (t < 2) l += s_red[ww][7 + t];
        }
        s_fin[t] = hi + l;
        if (t < 2) s_fin_lo[t] = l - (s_fin[t] - hi);
      }
      __syncthreads();
      if (t < 3) {  // lab dipole: mu = O mu', mu' = d dR (Re(S+ + S-), Im(S+ - S-), 2 Re Z)
        const float sc = (float)sp.dipole * sp.dR;
        const float lab =
            sc * (s_rot[3 * t] * s_fin[4] + s_rot[3 * t + 1] * s_fin[5] + s_rot[3 * t + 2] * s_fin[6]);
        const double nl = (double)lab;
        md.dmu[3 * (long long)m + t] = nl - s_mu[t];
        md.mu[3 * (long long)m + t] = nl;
      } else if (t < 5) {
        const double P = ((double)s_fin[t - 3] + (double)s_fin_lo[t - 3]) * (double)sp.dR;
        md.pop[2 * (long long)m + (t - 3)] = P;
        if (!isfinite(P)) atomicOr(err, kErrNonFinite);
      } else if (t < 7) {
        md.absorbed[2 * (long long)m + (t - 5)] = s_abs[t - 5] + (double)s_fin[t - 3] * (double)sp.dR;
      } else if (t == 7) {
        md.ncorr[m] = rounding_feedback(s_fin[7], s_fin[0] + s_fin[1]);
      }
    }
  }
}


}  // namespace

template <int J, int TILE>
static void launch_rspace_jt(const SpeciesDev& sp, const MolDev& md, int* err, const RspaceMaps& maps,
                             cudaStream_t s) {
  using D = RsDims<J, TILE>;
  launch_persistent(mol_rspace_kernel<J, TILE>, D::NT, D::BYTES, sp, md, err, maps, s);
}

template <int J>
static void launch_rspace_j(const SpeciesDev& sp, const MolDev& md, int* err, const RspaceMaps& maps,
                            int tile, cudaStream_t s) {
  if constexpr (J >= 9) {
    launch_rspace_jt<J, 8>(sp, md, err, maps, s);
  } else {
    if (tile == 16) launch_rspace_jt<J, 16>(sp, md, err, maps, s);
    else launch_rspace_jt<J, 32>(sp, md, err, maps, s);
  }
}

void launch_rspace(const SpeciesDev& sp, const MolDev& md, int* err, const RspaceMaps& maps, int tile,
                          cudaStream_t s) {
  switch (sp.jmax) {
    case 0: launch_rspace_j<0>(sp, md, err, maps, tile, s); break;
    case 1: launch_rspace_j<1>(sp, md, err, maps, tile, s); break;
    case 2: launch_rspace_j<2>(sp, md, err, maps, tile, s); break;
    case 3: launch_rspace_j<3>(sp, md, err, maps, tile, s); break;
    case 4: launch_rspace_j<4>(sp, md, err, maps, tile, s); break;
    case 5: launch_rspace_j<5>(sp, md, err, maps, tile, s); break;
    case 6: launch_rspace_j<6>(sp, md, err, maps, tile, s); break;
    case 7: launch_rspace_j<7>(sp, md, err, maps, tile, s); break;
    case 8: launch_rspace_j<8>(sp, md, err, maps, tile, s); break;
    case 9: launch_rspace_j<9>(sp, md, err, maps, tile, s); break;
    case 10: launch_rspace_j<10>(sp, md, err, maps, tile, s); break;
    case 11: launch_rspace_j<11>(sp, md, err, maps, tile, s); break;
    case 12: launch_rspace_j<12>(sp, md, err, maps, tile, s); break;
    case 13: launch_rspace_j<13>(sp, md, err, maps, tile, s); break;
    case 14: launch_rspace_j<14>(sp, md, err, maps, tile, s); break;
    case 15: launch_rspace_j<15>(sp, md, err, maps, tile, s); break;
    case 16: launch_rspace_j<16>(sp, md, err, maps, tile, s); break;
  }
}


cudaError_t upload_triplet_tables_tile(const CouplEntry* dip) { return upload_triplet_tables_local(dip); }

}  // namespace ms
