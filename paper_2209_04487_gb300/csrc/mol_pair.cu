// R-space pass with two radial points a thread (MS_KERN_PAIR): the kernels and
// their launch.  A translation unit of its own, so that it compiles beside
// mol.cu.
#include <cuda.h>
#include <cuda_fp16.h>
#include <cudaTypedefs.h>

#include <cstddef>
#include <type_traits>

#include "mol_common.cuh"

namespace ms {
namespace {

// ----------------------------------------------------------------------------
// R-space pass of the streaming form, tiled, two radial points per thread
// (MS_KERN_PAIR).  Tiles, tensor copies, persistence, bounded waits and the
// step computed are those of mol_rspace_kernel; here each thread holds a pair
// of neighbouring radial points of its rows, so the arithmetic runs as packed
// FP32x2 operations (one instruction for both points) and every shared-memory
// access moves 16 bytes.  Values whose complex products matter (eta, the
// series terms, the potential and mask tables) are kept per point pair as
// (Re p, Re p+1, Im p, Im p+1): a complex product is then four packed
// operations with no exchange of parts.  The state arrives and leaves as
// stored, (Re, Im) per point; the operations that keep real and imaginary
// parts apart (the update, its rounding residual, the sums, the dipole's
// real-coefficient couplings) run on it in that order.
//
// The coupling series is carried as R_n = M^n eta, with M = theta (E_perp X +
// E'_z Z) real in the turned frame, so no term needs the factor i: the sum
// S = sum_{n >= 1} (i^n / n!) R_n takes a real weight on even n and a weight
// times a swap of parts on odd n.  Rows are padded to whole warp slots (RPL
// rows of TILE / 2 threads); padded rows stay zero and are neither summed
// nor written.  PAR: the parity-reduced state (ground rows the even-j
// channels, excited rows the odd-j channels, each in channel order); the row
// table maps rows to channels and neighbour runs, so the arithmetic is the
// same.
// ----------------------------------------------------------------------------
constexpr int pair_rows(int slots, int rpw, int rpl) { return (slots + rpw - 1) / rpw * rpw * rpl; }
// rows per thread: 6 down to 3, the fewest padded rows (ties: more rows a thread)
constexpr int pair_rpw(int slots, int rpl) {
  int best = 6;
  for (int r = 5; r >= 3; --r)
    if (pair_rows(slots, r, rpl) < pair_rows(slots, best, rpl)) best = r;
  return best;
}

// One row of the pair kernel's row table (built per molecule); the
// coefficients appear twice, once per point of a pair.
struct RowP {
  float4 c0, c1, c2;  // theta x coupling: (u.x u.x u.y u.y) (u.z u.z d.x d.x) (d.y d.y d.z d.z) on the runs
  float4 ph;          // e^{i m phi_E}: (Re, Re, Im, Im)
  int ou, od, vo, pad;
};
// Dipole coefficients of a ground row, laid out as RowP's c0..c2 (built once per CTA).
struct DipP {
  float4 d0, d1, d2;
};

// rows of one surface in the parity-reduced layout: channels of j parity q up to J
constexpr int par_rows(int J, int q) {
  int n = 0;
  for (int j = q; j <= J; j += 2) n += 2 * j + 1;
  return n;
}

template <int J, int TILE, bool PAR = false>
struct Rs2Dims {
  static constexpr int NROT = (J + 1) * (J + 1), NV = 2 * (J + 1);
  static constexpr int NGR = PAR ? par_rows(J, 0) : NROT;       // ground rows
  static constexpr int ROWS = PAR ? NROT : 2 * NROT;             // stored rows
  static constexpr int TPR = TILE / 2, RPL = 32 / TPR;  // threads per row, rows per warp slot
  static constexpr int SLOTS = (ROWS + RPL - 1) / RPL;
  static constexpr int RPW = pair_rpw(SLOTS, RPL);
  static constexpr int NW = (SLOTS + RPW - 1) / RPW, NT = 32 * NW;
  static constexpr int RP = NW * RPW * RPL;  // rows with padding
  static constexpr bool EXACT = RP == ROWS;
  static constexpr int SEG = TILE * (int)sizeof(float2), SLOT = RPL * SEG;
  static constexpr int BOXR = ROWS < 256 ? ROWS : 256, NBOX = (ROWS + BOXR - 1) / BOXR;
  static constexpr int TBB = (kTriGuard + RP) * SEG;
  static constexpr int O_STG = 0, O_VD = O_STG + 2 * RP * SEG, O_VH = O_VD + 2 * NV * SEG;
  static constexpr int O_MK = O_VH + 2 * NV * SEG, O_TB = O_MK + (SEG < 128 ? 128 : SEG), O_RT = O_TB + 2 * TBB;
  static constexpr int O_DT = O_RT + RP * (int)sizeof(RowP);
  static constexpr int BYTES = 128 + O_DT + NGR * (int)sizeof(DipP);
  // parity-reduced kernels: as many resident CTAs (up to 3) as their shared memory allows (78.1 against
  // 81.0 ms a step on the nanohole workload at J = 8, two CTAs before)
  static constexpr int MINB_SMEM = 228 * 1024 / (BYTES + 2048);
  static constexpr int MINB = PAR ? (MINB_SMEM < 1 ? 1 : (MINB_SMEM > 3 ? 3 : MINB_SMEM))
                                  : (J >= 9 ? 1 : (TILE == 8 ? 3 : 2));
  static_assert(TILE == 8 || TILE == 16 || TILE == 32, "tile of 8, 16 or 32 radial points");
  static_assert(NT <= 1024 && BYTES <= 227 * 1024, "one CTA per molecule fits");
  static_assert(SLOT == 512, "a warp slot is 512 contiguous bytes");
  static_assert((RP * SEG) % 128 == 0 && (NV * SEG) % 128 == 0 && (NBOX == 1 || (BOXR * SEG) % 128 == 0) &&
                    O_RT % 16 == 0,
                "tensor-copy destinations 128-byte aligned, tables 16-byte aligned");
};

__device__ __forceinline__ float2 lo2(float4 v) { return make_float2(v.x, v.y); }
__device__ __forceinline__ float2 hi2(float4 v) { return make_float2(v.z, v.w); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 neg2(float2 a) { return make_float2(-a.x, -a.y); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __fadd2_rn(a, neg2(b)); }
// (ax + i ay)(bx + i by) on point pairs
__device__ __forceinline__ void cmul2(float2 ax, float2 ay, float2 bx, float2 by, float2& rx, float2& ry) {
  rx = fma2(ax, bx, neg2(mul2(ay, by)));
  ry = fma2(ax, by, mul2(ay, bx));
}
template <int OFF>
__device__ __forceinline__ float4 lds4(const unsigned char* base, int off) {
  return *reinterpret_cast<const float4*>(base + off + OFF);
}
template <int OFF>
__device__ __forceinline__ void sts4(unsigned char* base, int off, float4 v) {
  *reinterpret_cast<float4*>(base + off + OFF) = v;
}
// round_update on one point held as a (Re, Im) pair, packed: s' = fl(s + D'),
// D' = D + c s, with the exact residual of that rounding folded into acc
// (per part; the two parts are added at the end)
__device__ __forceinline__ float2 round_update2(float2 sv, float2 D, float2 c, float2& acc) {
  const float2 d = fma2(c, sv, D);
  const float2 n = add2(sv, d);
  const float2 b = sub2(n, sv);
  const float2 e = add2(sub2(sv, sub2(n, b)), sub2(d, b));
  acc = fma2(n, e, acc);
  return n;
}
// compensated sums of point pairs (TwoSum per part)
__device__ __forceinline__ void acc2p(float2& hi, float2& lo, float2 x) {
  const float2 t = add2(hi, x);
  const float2 z = sub2(t, hi);
  lo = add2(lo, add2(sub2(hi, sub2(t, z)), sub2(x, z)));
  hi = t;
}

// first row of shell j' within its surface (the surface holding j')
template <bool PAR>
__device__ __forceinline__ int shell_row(int jp) {
  if (!PAR) return jp * jp;
  int r = 0;
  for (int jj = jp & 1; jj < jp; jj += 2) r += 2 * jj + 1;
  return r;
}

template <int J, int TILE, bool PAR>
__global__ void __launch_bounds__(Rs2Dims<J, TILE, PAR>::NT, Rs2Dims<J, TILE, PAR>::MINB)
    mol_rspace_pair_kernel(SpeciesDev sp, MolDev md, int* err, const __grid_constant__ RspaceMaps maps) {
  using D = Rs2Dims<J, TILE, PAR>;
  constexpr int NROT = D::NGR, ROWS = D::ROWS, NV = D::NV, NW = D::NW, RPW = D::RPW, NT = D::NT;
  constexpr int RPL = D::RPL, SEG = D::SEG, SLOT = D::SLOT, TBB = D::TBB, G0 = kTriGuard * SEG;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ __align__(8) unsigned long long s_bar[1];
  __shared__ float s_rot[9];
  __shared__ double s_mu[3], s_abs[2];
  __shared__ float2 s_ph[2 * kMaxJ + 1];
  __shared__ float s_red[NW][10];
  __shared__ float s_fin[8], s_fin_lo[2];

  const int NR = sp.nr;
  const int t = threadIdx.x, lane = t & 31, w = t >> 5;
  const int part = lane / D::TPR, pp = lane % D::TPR;  // row within the warp slot, point pair
  const int pad = (int)((128u - (smem_u32(smem_raw) & 127u)) & 127u);
  unsigned char* const sm = smem_raw;
  // this thread's byte offsets: own rows RPL (w + NW i) + part at points 2 pp, 2 pp + 1
  const int own = pad + w * SLOT + lane * 16;
  const int rtw = pad + D::O_RT + (RPL * w + part) * (int)sizeof(RowP);
  const int dtw = pad + D::O_DT + (RPL * w + part) * (int)sizeof(DipP);
  auto issue = [&](int mol, int ck) {
    const int r0 = ck * TILE, b = ck & 1;
    unsigned char* base = sm + pad;
#pragma unroll
    for (int k = 0; k < D::NBOX; ++k) {
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
  constexpr unsigned kChunkBytes = (2 * ROWS + 2 * NV + 1) * SEG;
  const int nchunks = NR / TILE;  // even: NR is 64, 128 or 256

  int lm = blockIdx.x;
  if (t == 0) {
    mbar_init(&s_bar[0], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    mbar_expect_tx(&s_bar[0], kChunkBytes);
    issue(lm, 0);
  }
  // both term buffers zeroed once: the guard rows stay zero, and every row a
  // zero coefficient may read (the dipole reads only excited rows' s', so a
  // down-run at its lowest shell can land on ground rows never stored) holds
  // finite data from then on
  for (int q = t; q < 2 * TBB / 16; q += NT)
    reinterpret_cast<float4*>(sm + pad + D::O_TB)[q] = make_float4(0.f, 0.f, 0.f, 0.f);
  if constexpr (!D::EXACT) {  // padded staging rows: zero, and never written by the copies
    for (int q = t; q < (D::RP - ROWS) * TILE; q += NT) {
      reinterpret_cast<float2*>(sm + pad + D::O_STG + ROWS * SEG)[q] = make_float2(0.f, 0.f);
      reinterpret_cast<float2*>(sm + pad + D::O_STG + (D::RP + ROWS) * SEG)[q] = make_float2(0.f, 0.f);
    }
  }
  for (int q = t; q < NROT; q += NT) {  // dipole coefficients of the ground rows (the same for every molecule)
    int c = q;                           // channel of ground row q
    if constexpr (PAR) {
      int r = q, jj = 0;
      while (r >= 2 * jj + 1) { r -= 2 * jj + 1; jj += 2; }
      c = jj * jj + r;
    }
    const int j = j_of(c);
    const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
    const float4 du = j < J ? g_tri_up[c] : z4, dd = j > 0 ? g_tri_dn[c] : z4;
    DipP d;
    d.d0 = make_float4(du.x, du.x, du.y, du.y);
    d.d1 = make_float4(du.z, du.z, dd.x, dd.x);
    d.d2 = make_float4(dd.y, dd.y, dd.z, dd.z);
    *reinterpret_cast<DipP*>(sm + pad + D::O_DT + q * (int)sizeof(DipP)) = d;
  }
  auto ground = [&](int i) { return RPL * (w + NW * i) + part < NROT; };
  auto valid = [&](int i) { return D::EXACT || RPL * (w + NW * i) + part < ROWS; };

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
    const float2 cf2 = make_float2(cfix, cfix);
    __syncthreads();
    for (int q = t; q < D::RP; q += NT) {  // the row table of this molecule (padding: zero, guard rows)
      RowP r;
      if (!D::EXACT && q >= ROWS) {
        r.c0 = r.c1 = r.c2 = make_float4(0.f, 0.f, 0.f, 0.f);
        r.ph = make_float4(1.f, 1.f, 0.f, 0.f);
        r.ou = r.od = D::O_TB;
        r.vo = 0;
      } else {
        // theta E_perp / 2 on the X runs and theta E'_z on the Z runs (frame turned so E'_y = 0)
        const float ep = sqrtf(f.y * f.y + f.z * f.z), ez = f.x;
        const int sf = q >= NROT;
        int c = q - sf * NROT;  // channel of the row
        if constexpr (PAR) {    // surface sf holds the channels of j parity sf
          int r0 = c, jj = sf;
          while (r0 >= 2 * jj + 1) { r0 -= 2 * jj + 1; jj += 2; }
          c = jj * jj + r0;
        }
        const int j = j_of(c), mm = c - j * j - j;
        const int other = kTriGuard + (1 - sf) * NROT;  // first row of the other surface
        const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
        const float4 du = j < J ? g_tri_up[c] : z4, dd = j > 0 ? g_tri_dn[c] : z4;
        const float ux = ep * du.x, uy = ez * du.y, uz = ep * du.z;
        const float dx = ep * dd.x, dy = ez * dd.y, dz = ep * dd.z;
        r.c0 = make_float4(ux, ux, uy, uy);
        r.c1 = make_float4(uz, uz, dx, dx);
        r.c2 = make_float4(dy, dy, dz, dz);
        const float2 ph = s_ph[mm + J];
        r.ph = make_float4(ph.x, ph.x, ph.y, ph.y);
        // the runs (j +- 1, mm - 1 .. mm + 1) of the other surface start at its
        // rows of (j +- 1, mm - 1): shell start + (mm - 1) + (j +- 1)
        r.ou = D::O_TB + (j < J ? (other + shell_row<PAR>(j + 1) + mm + j) * SEG : 0);
        r.od = D::O_TB + (j > 0 ? (other + shell_row<PAR>(j - 1) + mm + j - 2) * SEG : 0);
        r.vo = (sf * (J + 1) + j) * SEG;
      }
      r.pad = 0;
      *reinterpret_cast<RowP*>(sm + pad + D::O_RT + q * (int)sizeof(RowP)) = r;
    }
    float4 sv[RPW], dv[RPW];  // s and d2 of the own rows, as stored: (Re, Im) of point 2 pp, then 2 pp + 1
    float2 sx[RPW], sy[RPW];  // the series sum S, pair layout
    float2 pg_hi = make_float2(0.f, 0.f), pg_lo = pg_hi, pe_hi = pg_hi, pe_lo = pg_hi;  // populations
    float2 a_g = pg_hi, a_e = pg_hi, aS = pg_hi, aZ = pg_hi, aD = pg_hi, rnd = pg_hi;
    float2* gs = sp.psi + (long long)lm * ROWS * NR;

    // R_n = M R_{n-1} from term buffer P, added to S with weight (ka, kb):
    // odd n (P = 0): S += i k R, ka = -k, kb = k; even n (P = 1): S += k R, kb = k
    auto term = [&](auto Pc, int n, float2 ka, float2 kb) {
      constexpr int P = decltype(Pc)::value;
      const bool store = n < nterms;
#pragma unroll
      for (int i = 0; i < RPW; ++i) {
        const unsigned char* rt = sm + rtw + NW * RPL * i * (int)sizeof(RowP);
        const float4 c0 = *reinterpret_cast<const float4*>(rt + offsetof(RowP, c0));
        const float4 c1 = *reinterpret_cast<const float4*>(rt + offsetof(RowP, c1));
        const float4 c2 = *reinterpret_cast<const float4*>(rt + offsetof(RowP, c2));
        const int2 oo = *reinterpret_cast<const int2*>(rt + offsetof(RowP, ou));
        const int ou = pad + pp * 16 + oo.x, od = pad + pp * 16 + oo.y;
        const float4 u0 = lds4<P * TBB>(sm, ou), u1 = lds4<P * TBB + SEG>(sm, ou),
                     u2 = lds4<P * TBB + 2 * SEG>(sm, ou);
        const float4 e0 = lds4<P * TBB>(sm, od), e1 = lds4<P * TBB + SEG>(sm, od),
                     e2 = lds4<P * TBB + 2 * SEG>(sm, od);
        float2 rx = mul2(lo2(c0), lo2(u0)), ry = mul2(lo2(c0), hi2(u0));
        rx = fma2(hi2(c0), lo2(u1), rx); ry = fma2(hi2(c0), hi2(u1), ry);
        rx = fma2(lo2(c1), lo2(u2), rx); ry = fma2(lo2(c1), hi2(u2), ry);
        rx = fma2(hi2(c1), lo2(e0), rx); ry = fma2(hi2(c1), hi2(e0), ry);
        rx = fma2(lo2(c2), lo2(e1), rx); ry = fma2(lo2(c2), hi2(e1), ry);
        rx = fma2(hi2(c2), lo2(e2), rx); ry = fma2(hi2(c2), hi2(e2), ry);
        if constexpr (P == 0) {
          sx[i] = fma2(ka, ry, sx[i]);
          sy[i] = fma2(kb, rx, sy[i]);
        } else {
          sx[i] = fma2(kb, rx, sx[i]);
          sy[i] = fma2(kb, ry, sy[i]);
        }
        if (store) sts4<(1 - P) * TBB + G0>(sm, own + D::O_TB + NW * i * SLOT, make_float4(rx.x, rx.y, ry.x, ry.y));
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
      const float4 mk = *reinterpret_cast<const float4*>(sm + pad + D::O_MK + pp * 16);  // (m, m, 1-m^2, 1-m^2)
      // ---- s, d2; eta = e^{i m phi} V^{1/2} u into term buffer 0 (pair layout)
#pragma unroll
      for (int i = 0; i < RPW; ++i) {
        sv[i] = lds4<D::O_STG>(sm, own + NW * i * SLOT);
        dv[i] = lds4<D::O_STG + D::RP * SEG>(sm, own + NW * i * SLOT);
        sx[i] = sy[i] = make_float2(0.f, 0.f);
        if (nterms > 0) {
          const unsigned char* rt = sm + rtw + NW * RPL * i * (int)sizeof(RowP);
          const int vo = pad + pp * 16 + *reinterpret_cast<const int*>(rt + offsetof(RowP, vo));
          const float4 vh = lds4<OVH>(sm, vo);
          const float4 ph = *reinterpret_cast<const float4*>(rt + offsetof(RowP, ph));
          const float2 ux = make_float2(sv[i].x + dv[i].x, sv[i].z + dv[i].z);
          const float2 uy = make_float2(sv[i].y + dv[i].y, sv[i].w + dv[i].w);
          float2 ax, ay, ex, ey;
          cmul2(lo2(vh), hi2(vh), ux, uy, ax, ay);
          cmul2(lo2(ph), hi2(ph), ax, ay, ex, ey);
          sts4<D::O_TB + G0>(sm, own + NW * i * SLOT, make_float4(ex.x, ex.y, ey.x, ey.y));
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
      float fac = 1.f;  // 1 / n!
      for (int n = 1; n <= nterms; n += 2) {
        fac /= (float)n;
        const float k1 = (n & 2) ? -fac : fac;  // i^n / n! = i k1
        term(std::integral_constant<int, 0>(), n, make_float2(-k1, -k1), make_float2(k1, k1));
        if (n + 1 <= nterms) {
          fac /= (float)(n + 1);
          const float k2 = ((n + 1) & 2) ? -fac : fac;  // i^(n+1) / (n+1)! = k2
          term(std::integral_constant<int, 1>(), n + 1, make_float2(0.f, 0.f), make_float2(k2, k2));
        }
      }
      // ---- d1 = (V - 1) u + V^{1/2} e^{-i m phi} S ; mask ; s' = s + (d2 + d1) + cfix s
      const int sbo = (nterms & 1) * TBB;  // s' buffer: not read by the last term
      float2* gsw = gs + (long long)(RPL * w + part) * NR + ck * TILE + 2 * pp;
      const bool masked = mk.x < 1.f || mk.y < 1.f;
#pragma unroll
      for (int i = 0; i < RPW; ++i) {
        const unsigned char* rt = sm + rtw + NW * RPL * i * (int)sizeof(RowP);
        const int vo = pad + pp * 16 + *reinterpret_cast<const int*>(rt + offsetof(RowP, vo));
        const float2 ux = make_float2(sv[i].x + dv[i].x, sv[i].z + dv[i].z);
        const float2 uy = make_float2(sv[i].y + dv[i].y, sv[i].w + dv[i].w);
        const float4 vd = lds4<OVD>(sm, vo);
        float2 d1x, d1y;
        cmul2(lo2(vd), hi2(vd), ux, uy, d1x, d1y);
        if (nterms > 0) {
          const float4 vh = lds4<OVH>(sm, vo);
          const float4 ph = *reinterpret_cast<const float4*>(rt + offsetof(RowP, ph));
          // conj(ph) S, then V^{1/2} times it
          const float2 tx = fma2(lo2(ph), sx[i], mul2(hi2(ph), sy[i]));
          const float2 ty = fma2(lo2(ph), sy[i], neg2(mul2(hi2(ph), sx[i])));
          d1x = fma2(lo2(vh), tx, fma2(neg2(hi2(vh)), ty, d1x));
          d1y = fma2(lo2(vh), ty, fma2(hi2(vh), tx, d1y));
        }
        const bool gr = ground(i);
        if (masked) {
          const float2 mv = lo2(mk), mm1 = make_float2(mk.x - 1.f, mk.y - 1.f);
          const float2 px = add2(ux, d1x), py = add2(uy, d1y);
          d1x = fma2(mm1, ux, mul2(mv, d1x));
          d1y = fma2(mm1, uy, mul2(mv, d1y));
          const float2 dd = mul2(hi2(mk), fma2(px, px, mul2(py, py)));
          if (gr) a_g = add2(a_g, dd);
          else a_e = add2(a_e, dd);
        }
        // back to (Re, Im) per point: D = d2 + d1
        const float2 D0 = make_float2(dv[i].x + d1x.x, dv[i].y + d1y.x);
        const float2 D1 = make_float2(dv[i].z + d1x.y, dv[i].w + d1y.y);
        const float2 n0 = round_update2(lo2(sv[i]), D0, cf2, rnd);
        const float2 n1 = round_update2(hi2(sv[i]), D1, cf2, rnd);
        const float4 sn = make_float4(n0.x, n0.y, n1.x, n1.y);
        if (valid(i)) *reinterpret_cast<float4*>(gsw + (long long)(RPL * NW * i) * NR) = sn;
        if (!gr) sts4<D::O_TB + G0>(sm, own + sbo + NW * i * SLOT, sn);  // the dipole reads excited rows only
        sv[i] = sn;
        const float2 b2 = make_float2(fmaf(n0.x, n0.x, n0.y * n0.y), fmaf(n1.x, n1.x, n1.y * n1.y));
        if (gr) acc2p(pg_hi, pg_lo, b2);  // compensated from the first term on
        else acc2p(pe_hi, pe_lo, b2);
      }
      __syncthreads();
      // ---- dipole in the molecule frame on s' (as stored): sum_c conj(g_c) (A e)_c for A = Z, S+, S-
#pragma unroll
      for (int i = 0; i < RPW; ++i) {
        if (ground(i)) {
          const unsigned char* rt = sm + rtw + NW * RPL * i * (int)sizeof(RowP);
          const unsigned char* dt = sm + dtw + NW * RPL * i * (int)sizeof(DipP);
          const float4 q0 = *reinterpret_cast<const float4*>(dt + offsetof(DipP, d0));
          const float4 q1 = *reinterpret_cast<const float4*>(dt + offsetof(DipP, d1));
          const float4 q2 = *reinterpret_cast<const float4*>(dt + offsetof(DipP, d2));
          const int2 oo = *reinterpret_cast<const int2*>(rt + offsetof(RowP, ou));
          const int a = pad + pp * 16 + oo.x + sbo, c = pad + pp * 16 + oo.y + sbo;
          const float4 u0 = lds4<0>(sm, a), u1 = lds4<SEG>(sm, a), u2 = lds4<2 * SEG>(sm, a);
          const float4 e0 = lds4<0>(sm, c), e1 = lds4<SEG>(sm, c), e2 = lds4<2 * SEG>(sm, c);
#pragma unroll
          for (int h = 0; h < 2; ++h) {  // the two points, (Re, Im) each
            const float2 g = h ? hi2(sv[i]) : lo2(sv[i]);
            const float2 U0 = h ? hi2(u0) : lo2(u0), U1 = h ? hi2(u1) : lo2(u1), U2 = h ? hi2(u2) : lo2(u2);
            const float2 E0 = h ? hi2(e0) : lo2(e0), E1 = h ? hi2(e1) : lo2(e1), E2 = h ? hi2(e2) : lo2(e2);
            const float2 wP = fma2(lo2(q0), U0, mul2(hi2(q1), E0));  // S+ from both runs
            const float2 wZ = fma2(hi2(q0), U1, mul2(lo2(q2), E1));  // Z
            const float2 wM = fma2(lo2(q1), U2, mul2(hi2(q2), E2));  // S-
            aS = fma2(g, add2(wP, wM), aS);            // (sum gx (P+M)x, sum gy (P+M)y)
            aZ = fma2(g, wZ, aZ);
            aD = fma2(make_float2(g.y, g.x), sub2(wP, wM), aD);  // (sum gy (P-M)x, sum gx (P-M)y)
          }
        }
      }
      return true;
    };

    for (int ck = 0; ck < nchunks; ck += 2) {
      if (!chunk(std::integral_constant<int, 0>(), ck)) return;
      if (!chunk(std::integral_constant<int, 1>(), ck + 1)) return;
    }
    // ---- block reduction: populations compensated, the rest plain FP32
    {
      float v[8], lo[2];
      v[0] = pg_hi.x; lo[0] = pg_lo.x + pg_lo.y; acc2(v[0], lo[0], pg_hi.y);
      v[1] = pe_hi.x; lo[1] = pe_lo.x + pe_lo.y; acc2(v[1], lo[1], pe_hi.y);
      v[2] = a_g.x + a_g.y;
      v[3] = a_e.x + a_e.y;
      v[4] = aS.x + aS.y;         // Re(P + M)
      v[5] = aD.y - aD.x;         // Im(P - M)
      v[6] = 2.f * (aZ.x + aZ.y); // 2 Re Z
      v[7] = rnd.x + rnd.y;
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
static void launch_pair_jt(const SpeciesDev& sp, const MolDev& md, int* err, const RspaceMaps& maps,
                           cudaStream_t s) {
  // the parity-reduced kernels exist from J = 5 on at the rule's tile width
  constexpr bool kPar = J >= 5 && TILE == (J >= 9 ? 8 : 16);
  if constexpr (kPar) {
    if (sp.par) {
      using P = Rs2Dims<J, TILE, true>;
      launch_persistent(mol_rspace_pair_kernel<J, TILE, true>, P::NT, P::BYTES, sp, md, err, maps, s);
      return;
    }
  }
  using D = Rs2Dims<J, TILE, false>;
  launch_persistent(mol_rspace_pair_kernel<J, TILE, false>, D::NT, D::BYTES, sp, md, err, maps, s);
}

void launch_rspace_pair(const SpeciesDev& sp, const MolDev& md, int* err, const RspaceMaps& maps, int tile,
                               cudaStream_t s) {
#define MS_PAIR_LO(J)                                                  \
  case J:                                                              \
    if (tile == 16) launch_pair_jt<J, 16>(sp, md, err, maps, s);       \
    else launch_pair_jt<J, 32>(sp, md, err, maps, s);                  \
    break;
#define MS_PAIR_HI(J)                                                  \
  case J:                                                              \
    if (tile == 8) launch_pair_jt<J, 8>(sp, md, err, maps, s);         \
    else launch_pair_jt<J, 16>(sp, md, err, maps, s);                  \
    break;
#define MS_PAIR_8(J)                                                   \
  case J:                                                              \
    launch_pair_jt<J, 8>(sp, md, err, maps, s);                        \
    break;
  switch (sp.jmax) {
    MS_PAIR_LO(0) MS_PAIR_LO(1) MS_PAIR_LO(2) MS_PAIR_LO(3) MS_PAIR_LO(4)
    MS_PAIR_HI(5) MS_PAIR_HI(6) MS_PAIR_HI(7) MS_PAIR_HI(8)
    MS_PAIR_8(9) MS_PAIR_8(10) MS_PAIR_8(11) MS_PAIR_8(12) MS_PAIR_8(13) MS_PAIR_8(14) MS_PAIR_8(15) MS_PAIR_8(16)
  }
#undef MS_PAIR_LO
#undef MS_PAIR_HI
#undef MS_PAIR_8
}


cudaError_t upload_triplet_tables_pair(const CouplEntry* dip) { return upload_triplet_tables_local(dip); }

}  // namespace ms
