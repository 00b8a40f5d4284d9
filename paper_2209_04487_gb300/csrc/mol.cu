// Molecular split-operator step (Eqs. 3-5 with the surfaces of Eqs. 6-7),
// one CTA per molecule, the molecule's whole state resident in shared memory.
//
// The library stores s = T^{-1/2} psi, so that one coupled step is
//   u  = T s                                   (kinetic pass, per channel)
//   s' = Mask V^{1/2} K(E') V^{1/2} u          (R-space pass, per radial point)
// which equals the paper's split-operator step T^{1/2} Mask V^{1/2} K V^{1/2}
// T^{1/2} on psi (T commutes with the angular coupling because the
// transition dipole is R-independent, and is unitary per channel, so
// populations and the dipole can be taken from s').
//
// Norm-preserving FP32 arithmetic: every unit-modulus factor (potential
// phase, kinetic phase, FFT twiddle) is carried as an FP32 hi+lo pair and
// applied with a compensated product, so the factor is exact to ~1e-15 and
// only unbiased output rounding remains.  Every factor of the step is close
// to the identity (|V dtau| and |k^2 dtau/2mu| are a few 1e-2 at one
// molecular step per field step, O(1) under sub-stepping), so the step is
// computed as a correction: d2 = (T - 1) s, u = s + d2,
// d1 = (V - 1) u + V^{1/2} S with S = sum_{n>=1} (i theta sigma_x M)^n/n!
// V^{1/2} u (Taylor series of the coupling exponential, |theta M| << 1), and
// s' = s + (d2 + d1): the full-magnitude state is rounded once per step,
// which turns the FP32 norm error from a drift into a random walk of about
// 1e-8 per step.  That one rounding's exact residual (TwoSum) gives the norm
// it changed; the next step scales its update by the factor that returns it
// (round_update), so the walk of the final roundings does not accumulate:
// what remains is one step's rounding plus the much smaller rounding inside
// the correction.  The coupling is evaluated in the frame turned about
// z that puts E' in the xz plane (a diagonal phase on the correction only),
// where M is real.
#include <cuda.h>
#include <cuda_fp16.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cmath>
#include <cstddef>
#include <mutex>
#include <type_traits>
#include <vector>

#include "ms_internal.cuh"
#include "mol_common.cuh"

namespace ms {

namespace {

constexpr int kPad = 0;  // state rows are stored unpadded (one bulk copy per molecule)

template <int NR>
struct FFTShape;
template <>
struct FFTShape<64> {
  static constexpr int N1 = 8, N2 = 8, THREADS = 256;
};
template <>
struct FFTShape<128> {
  static constexpr int N1 = 16, N2 = 8, THREADS = 256;
};
template <>
struct FFTShape<256> {
  static constexpr int N1 = 16, N2 = 16, THREADS = 256;
};

// cos / sin of t*pi/8, t = 0..7 (exact decimal expansions of the constants)
__host__ __device__ constexpr double cos_pi8(int t) {
  return t == 0 ? 1.0
       : t == 1 ? 0.92387953251128675613
       : t == 2 ? 0.70710678118654752440
       : t == 3 ? 0.38268343236508977173
       : t == 4 ? 0.0
       : t == 5 ? -0.38268343236508977173
       : t == 6 ? -0.70710678118654752440
                : -0.92387953251128675613;
}
__host__ __device__ constexpr double sin_pi8(int t) { return t <= 4 ? cos_pi8(4 - t) : cos_pi8(t - 4); }
__host__ __device__ constexpr float hi_of(double v) { return (float)v; }
__host__ __device__ constexpr float lo_of(double v) { return (float)(v - (double)(float)v); }

// (x) * (c + i s) with c = ch + cl, s = sh + sl (compensated)
__device__ __forceinline__ float2 cmul_c(float2 x, float ch, float sh, float cl, float sl) {
  const float re_lo = fmaf(x.x, cl, -x.y * sl);
  const float im_lo = fmaf(x.x, sl, x.y * cl);
  return make_float2(fmaf(x.x, ch, fmaf(-x.y, sh, re_lo)), fmaf(x.x, sh, fmaf(x.y, ch, im_lo)));
}
// same, plus an addend folded into the last rounding
__device__ __forceinline__ float2 cmul_c_add(float2 x, float4 w, float2 a) {
  const float re_lo = fmaf(x.x, w.z, fmaf(-x.y, w.w, a.x));
  const float im_lo = fmaf(x.x, w.w, fmaf(x.y, w.z, a.y));
  return make_float2(fmaf(x.x, w.x, fmaf(-x.y, w.y, re_lo)), fmaf(x.x, w.y, fmaf(x.y, w.x, im_lo)));
}

// multiply by exp(-+ i t pi/8) (forward: minus)
template <int T, bool INV>
__device__ __forceinline__ float2 twiddle16(float2 v) {
  if constexpr (T == 0) {
    return v;
  } else if constexpr (T == 4) {
    return INV ? make_float2(-v.y, v.x) : make_float2(v.y, -v.x);
  } else {
    constexpr float c = (float)cos_pi8(T);
    constexpr float s = INV ? (float)sin_pi8(T) : -(float)sin_pi8(T);
    return make_float2(fmaf(v.x, c, -v.y * s), fmaf(v.x, s, v.y * c));
  }
}

template <int L>
__device__ constexpr int bitrev(int a) {
  int r = 0;
  for (int b = 1, q = L >> 1; b < L; b <<= 1, q >>= 1)
    if (a & b) r |= q;
  return r;
}

// In-register DFT of size L (8 or 16), radix-2 decimation in time.
template <int L, bool INV, int H, int J>
__device__ __forceinline__ void dft_stage_j(float2 (&x)[L]) {
  if constexpr (J < H) {
    constexpr int T = J * (16 / (2 * H));
#pragma unroll
    for (int a = J; a < L; a += 2 * H) {
      const float2 u = x[a];
      const float2 v = twiddle16<T, INV>(x[a + H]);
      x[a] = u + v;
      x[a + H] = u - v;
    }
    dft_stage_j<L, INV, H, J + 1>(x);
  }
}
template <int L, bool INV, int H>
__device__ __forceinline__ void dft_stages(float2 (&x)[L]) {
  if constexpr (H < L) {
    dft_stage_j<L, INV, H, 0>(x);
    dft_stages<L, INV, 2 * H>(x);
  }
}
template <int L, bool INV>
__device__ __forceinline__ void dft_reg(float2 (&x)[L]) {
#pragma unroll
  for (int a = 0; a < L; ++a) {
    const int b = bitrev<L>(a);
    if (b > a) {
      const float2 t = x[a];
      x[a] = x[b];
      x[b] = t;
    }
  }
  dft_stages<L, INV, 1>(x);
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Four-step FFT pass on all `rows` rows (each NR complex, stride NRP) held
// in shared memory, in place: forward DFT, multiply by kph[k], inverse DFT.
// With kph = (P_k - 1)/NR it produces (T - 1) x; with kph = P_k/NR it
// applies T.  n = n1 + N1 n2, k = k2 + N2 k1.  Step A: per n1, an N2-point
// DFT over n2 and the twiddle exp(-2 pi i n1 k2/NR); step B: per k2, an
// N1-point DFT over n1.  The intermediate y[n1][k2] lives at n1 + N1 k2,
// xor-swizzled within each block of N1 so that step B is conflict free.
// Position of y[n1][k2] of `row` within the row: the xor with (k2 mod N1)
// spreads step B's N2 threads over distinct banks, the xor with CR for odd
// rows keeps the two rows that share a half-warp apart.
template <int N1, int N2>
__device__ __forceinline__ int swz(int n1, int k2, int row) {
  constexpr int CR = N1 > N2 ? N2 : (N1 == N2 && N1 == 8 ? 1 : 0);
  return (n1 ^ (k2 % N1) ^ ((row & 1) * CR)) + N1 * k2;
}

template <int NR>
__device__ void kinetic_pass(float2* st, int rows, const float2* kph, const float2* tw) {
  using S = FFTShape<NR>;
  constexpr int N1 = S::N1, N2 = S::N2, NT = S::THREADS, NRP = NR + kPad;
  const int t = threadIdx.x;
  {  // step A
    constexpr int per = NT / N1;
    const int n1 = t % N1, rsub = t / N1;
    for (int r0 = 0; r0 < rows; r0 += per) {
      const int row = r0 + rsub;
      float2 x[N2];
      if (row < rows) {
#pragma unroll
        for (int n2 = 0; n2 < N2; ++n2) x[n2] = st[row * NRP + n1 + N1 * n2];
      }
      __syncwarp();  // a row's N1 threads sit in one warp
      if (row < rows) {
        dft_reg<N2, false>(x);
#pragma unroll
        for (int k2 = 0; k2 < N2; ++k2)
          st[row * NRP + swz<N1, N2>(n1, k2, row)] = cmul(x[k2], tw[k2 * N1 + n1]);
      }
      __syncwarp();
    }
  }
  __syncthreads();
  {  // step B, the phase, inverse step B (in place per thread)
    constexpr int per = NT / N2;
    const int k2 = t % N2, rsub = t / N2;
    for (int r0 = 0; r0 < rows; r0 += per) {
      const int row = r0 + rsub;
      if (row < rows) {
        float2 x[N1];
#pragma unroll
        for (int n1 = 0; n1 < N1; ++n1) x[n1] = st[row * NRP + swz<N1, N2>(n1, k2, row)];
        dft_reg<N1, false>(x);  // x[k1] = X[k2 + N2 k1]
#pragma unroll
        for (int k1 = 0; k1 < N1; ++k1) x[k1] = cmul(x[k1], kph[k2 + N2 * k1]);
        dft_reg<N1, true>(x);
#pragma unroll
        for (int n1 = 0; n1 < N1; ++n1) st[row * NRP + swz<N1, N2>(n1, k2, row)] = x[n1];
      }
    }
  }
  __syncthreads();
  {  // inverse step A
    constexpr int per = NT / N1;
    const int n1 = t % N1, rsub = t / N1;
    for (int r0 = 0; r0 < rows; r0 += per) {
      const int row = r0 + rsub;
      float2 x[N2];
      if (row < rows) {
#pragma unroll
        for (int k2 = 0; k2 < N2; ++k2) {
          const float2 w = tw[k2 * N1 + n1];
          x[k2] = cmul(st[row * NRP + swz<N1, N2>(n1, k2, row)], make_float2(w.x, -w.y));
        }
        dft_reg<N2, true>(x);
      }
      __syncwarp();
      if (row < rows) {
#pragma unroll
        for (int n2 = 0; n2 < N2; ++n2) st[row * NRP + n1 + N1 * n2] = x[n2];
      }
      __syncwarp();
    }
  }
  __syncthreads();
}

// 16-byte asynchronous global -> shared copies (per thread), completed by
// cp.async.wait_group.
__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

__device__ __forceinline__ void load_state(float2* st, const float2* g, int rows, int NR, int NRP) {
  const float4* g4 = reinterpret_cast<const float4*>(g);
  const int per_row = NR / 2;
  const int total = rows * per_row;
  for (int q = threadIdx.x; q < total; q += blockDim.x) {
    const int row = q / per_row, col = q - row * per_row;
    reinterpret_cast<float4*>(st + row * NRP)[col] = g4[q];
  }
}


}  // namespace

// Angular coupling tables, shared by every species (they depend only on the
// channel (j, m), and a species with jmax < kMaxJ ignores entries whose
// neighbour lies beyond its basis).  c_rot: rows of Ex' X + Ez' Z written in
// the frame turned about z so that E'_y = 0 (kind 1: X entry, scaled by
// E_perp; kind 0: Z entry, scaled by E'_z).  c_dip: rows of Z (kind 0),
// S+ = sin(t)e^{ip} (kind 1) and S- (kind 2) for the dipole.
__constant__ CouplEntry c_rot[kMaxRot * kMaxCoupl];
__constant__ CouplEntry c_dip[kMaxRot * kMaxCoupl];

cudaError_t upload_coupling_tables(const CouplEntry* rot, const CouplEntry* dip) {
  cudaError_t e = cudaMemcpyToSymbol(c_rot, rot, sizeof(CouplEntry) * kMaxRot * kMaxCoupl);
  if (e != cudaSuccess) return e;
  return cudaMemcpyToSymbol(c_dip, dip, sizeof(CouplEntry) * kMaxRot * kMaxCoupl);
}

// Terms N of the coupling series exp(iA) ~ sum_{n <= N} (iA)^n / n!, for a
// Hermitian A with |A| <= x (x = theta |E'|).  Truncated after N terms the
// step changes the norm by up to 2 x^(N+1)/(N+1)! when N is odd; when N is
// even the first omitted term (iA)^(N+1) is odd in A and has no real part,
// so the norm changes only by up to 2 x^(N+2)/(N+1)!, while the amplitude
// the omitted terms carry, relative to the first-order term, is x^N/(N+1)!.
// N is the smallest count with a norm change below 1e-11 per step (1e-7 over
// 10^4 steps) and, for even N, an amplitude error below 1e-6.  24 flags a
// field out of range.
__device__ __forceinline__ int coupling_terms(float x) {
  if (!(x > 0.f)) return 0;
  float t = x;  // x^N / N!
  for (int N = 1; N < 24; ++N) {
    const float t1 = t * x / (float)(N + 1);  // x^(N+1) / (N+1)!
    const bool done = (N & 1) ? 2.f * t1 < 1e-11f : (2.f * t1 * x < 1e-11f && t1 < 1e-6f * x);
    if (done) return N;
    t = t1;
  }
  return 24;
}

// Local field at molecule m in its own frame (a.u.): fld = (E_perp, E'_z), the
// phases e^{i m' phi_E} (ph[m' + J], m' = -J..J) of the frame turned about z
// so that E'_y = 0, and the number of coupling-series terms (coupling_terms).
// Run by one thread.
__device__ __noinline__ void molecule_field(const MolDev& md, const Grid& g, int prescribed, int m, int J,
                                            double theta, float* fld, float2* ph, int* nterms, int* err) {
  float E[3];
  lab_field(md, g, prescribed, m, E, err);
  const float* O = md.rot + 9 * (long long)m;  // molecule -> lab, row-major
  const float inv_fau = 1.0f / 5.14220674763e11f;
  float Ep[3];
#pragma unroll
  for (int i = 0; i < 3; ++i) Ep[i] = (O[i] * E[0] + O[3 + i] * E[1] + O[6 + i] * E[2]) * inv_fau;
  const float eperp = sqrtf(Ep[0] * Ep[0] + Ep[1] * Ep[1]);
  fld[0] = eperp;
  fld[1] = Ep[2];
  // e^{i phi_E} = (E'_x + i E'_y)/E_perp; e^{i m phi_E} by repeated products
  const float2 e1 = eperp > 0.f ? make_float2(Ep[0] / eperp, Ep[1] / eperp) : make_float2(1.f, 0.f);
  float2 pw = make_float2(1.f, 0.f);
  ph[J] = pw;
  for (int q = 1; q <= J; ++q) {
    pw = cmul(pw, e1);
    ph[J + q] = pw;
    ph[J - q] = make_float2(pw.x, -pw.y);
  }
  const float x = (float)theta * sqrtf(eperp * eperp + Ep[2] * Ep[2]);
  if (!isfinite(x)) atomicOr(err, kErrNonFinite);  // a non-finite local field
  const int nt = coupling_terms(x);
  if (nt >= 24 || x > 4.f) atomicOr(err, kErrCouplingSeries);
  *nterms = nt;
}

constexpr int kChunk = 32;            // widest R-space chunk (one radial point per lane)

// ----------------------------------------------------------------------------
// the coupled molecular step, s = T^{-1/2} psi stored:
//   d2 = (T - 1) s           (kinetic pass, in shared memory)
//   u  = s + d2 = T s        (per radial point)
//   s' = Mask V^{1/2} K(E') V^{1/2} u, computed as s + (d2 + d1)
// ----------------------------------------------------------------------------
// FUSED: the whole state is staged in shared memory and the kinetic pass runs
// in this kernel.  Otherwise (streaming form) d2 = (T - 1) s comes from the
// scratch written by mol_kinetic_kernel and is streamed chunk by chunk with s.
// MAXR bounds the rows a thread owns in the R-space pass.
template <int NR, bool FUSED, int MAXR>
__global__ void __launch_bounds__(FFTShape<NR>::THREADS, FUSED ? 2 : (MAXR <= 4 ? 4 : (MAXR <= 12 ? 2 : 1)))
    mol_step_kernel(SpeciesDev sp, MolDev md, Grid g, int prescribed, int CH, int* err) {
  // CH radial points per chunk (32 down to 4): a warp covers 32/CH rows of CH points
  constexpr int NT = FFTShape<NR>::THREADS, NRP = NR + kPad, NW = NT / 32;
  extern __shared__ float4 smem4[];
  const int nrot = sp.nrot, rows = 2 * nrot, J = sp.jmax;
  float2* s_tw = reinterpret_cast<float2*>(smem4);      // [N2][N1] twiddles (fused)
  float2* s_kd = s_tw + (FUSED ? NR : 0);                // [NR] kinetic deltas (fused)
  float2* st = s_kd + (FUSED ? NR : 0);                  // [rows][NRP] state, then d2 (fused)
  float2* bY = st + (FUSED ? rows * NRP : 0);            // [rows][CH] Taylor terms / new state
  float2* bZ = bY + rows * CH;                           // [rows][CH] Taylor terms
  // per chunk, double buffered: old state [rows][CH], (streaming: d2
  // [rows][CH]), e^{-iV dtau} - 1 and e^{-iV dtau/2} [2(J+1)][CH] each, and
  // absorber mask [CH].  The half-step phase is read from its exact table:
  // with sub-stepping |V dtau| reaches O(1), where no short series of the
  // full-step delta would keep the coupling correction unitary.
  const int nd = FUSED ? 0 : rows;
  const int cbuf = (rows + nd + 4 * (J + 1) + 1) * CH;
  float2* bC = bZ + rows * CH;
  int2* s_prog = reinterpret_cast<int2*>(bC + 2 * cbuf);  // [nrot][6] (nbr*CH, coupling) this step
  int2* s_dipp = s_prog + nrot * kMaxCoupl;              // [nrot][6] (nbr*CH, dipole coefficient)
  int2* s_rinfo = s_dipp + nrot * kMaxCoupl;             // [rows] (table row, m + J)
  __shared__ __align__(8) unsigned long long s_bar[1];   // the state copy
  __shared__ float s_rot[9];                             // molecule -> lab rotation
  __shared__ double s_mu[3];                             // lab dipole of the previous step
  __shared__ double s_abs[2];                            // absorbed norm so far
  __shared__ float2 s_ph[2 * kMaxJ + 1];                 // e^{+i m phi_E}
  __shared__ float s_fld[2];                             // E_perp, E'_z (a.u.)
  __shared__ int s_nterms;
  __shared__ float2 s_red[NW][8];
  __shared__ float s_fin[8], s_fin_lo[8];

  const int t = threadIdx.x, lane = t & 31, w = t >> 5;
  const int LPR = 32 / CH;                       // row groups per warp
  const int rl = lane & (CH - 1), rg = lane / CH;
  const int row0 = w * LPR + rg, rstep = NW * LPR;
  const int lm = blockIdx.x;
  const int m = sp.mol[lm];
  float2* gs = sp.psi + (long long)lm * rows * NR;

  // chunk copy: old state, potential phases and mask of radial points [r0, r0 + CH)
  // every thread copies 16-byte pieces (cp.async); rows: old state, then
  // the potential deltas, the half-step phases, then the mask
  const float2* gd = FUSED ? nullptr : sp.d2 + (long long)lm * rows * NR;
  const int cp_per_row = CH / 2;                   // 16-byte pieces per chunk row
  const int cp_c2 = 2 * (t % cp_per_row), cp_q0 = t / cp_per_row, cp_qs = NT / cp_per_row;
  auto issue_chunk = [&](int r0, int b) {
    float2* buf = bC + b * cbuf;
    const int nv = 2 * (J + 1), nq = rows + nd + 2 * nv + 1;
    for (int q = cp_q0; q < nq; q += cp_qs) {
      const float2* src;
      if (q < rows) src = gs + (long long)q * NR;
      else if (q < rows + nd) src = gd + (long long)(q - rows) * NR;
      else if (q < rows + nd + nv) src = sp.vdelta + (long long)(q - rows - nd) * NR;
      else if (q < rows + nd + 2 * nv) src = sp.vhalf + (long long)(q - rows - nd - nv) * NR;
      else src = sp.maskw;
      cp_async16(buf + q * CH + cp_c2, src + r0 + cp_c2);
    }
    cp_async_commit();
  };
  if (t == 0) {
    mbar_init(&s_bar[0], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  if (FUSED && t == 0) {  // the whole (contiguous) state in one bulk copy
    mbar_expect_tx(&s_bar[0], (unsigned)(rows * NR * sizeof(float2)));
    bulk_g2s(st, gs, (unsigned)(rows * NR * sizeof(float2)), &s_bar[0]);
  }
  issue_chunk(0, 0);
  if (t < 9) s_rot[t] = md.rot[9 * (long long)m + t];
  else if (t < 12) s_mu[t - 9] = md.mu[3 * (long long)m + (t - 9)];
  else if (t < 14) s_abs[t - 12] = md.absorbed[2 * (long long)m + (t - 12)];
  if (FUSED) {
    for (int q = t; q < NR; q += NT) {
      s_tw[q] = __ldg(&sp.twiddle[q]);
      s_kd[q] = __ldg(&sp.kdelta[q]);
    }
  }
  for (int q = t; q < rows; q += NT) {
    const int sf = q >= nrot, c = q - sf * nrot, j = j_of(c);
    s_rinfo[q] = make_int2((sf * (J + 1) + j) * CH, c - j * j - j + J);
  }
  for (int q = t; q < nrot * kMaxCoupl; q += NT) {  // dipole rows: slots 0-1 Z, 2-3 S+, 4-5 S-
    const CouplEntry e = c_dip[q];
    const bool ok = (unsigned)e.nbr < (unsigned)nrot;
    s_dipp[q] = make_int2(ok ? e.nbr * CH : 0, __float_as_int(ok ? e.coef : 0.f));
  }

  // ---- local field, rotated into the molecule frame (a.u.)
  if (t == 0) molecule_field(md, g, prescribed, m, J, sp.theta, s_fld, s_ph, &s_nterms, err);
  __syncthreads();
  {  // this step's coupling rows: slots 0-1 Z (times E'_z), 2-5 X (times E_perp)
    const float eperp = s_fld[0], ez = s_fld[1];
    for (int q = t; q < nrot * kMaxCoupl; q += NT) {
      const CouplEntry e = c_rot[q];
      const bool ok = (unsigned)e.nbr < (unsigned)nrot;
      const float cf = ok ? e.coef * ((q % kMaxCoupl) >= 2 ? eperp : ez) : 0.f;
      s_prog[q] = make_int2(ok ? e.nbr * CH : 0, __float_as_int(cf));
    }
  }
  if (FUSED) {
    const bool ok = mbar_wait(&s_bar[0], 0, kWaitPolls);
    if (!__syncthreads_and(ok)) {  // uniform decision; copies still in flight get a second bounded wait
      if (t == 0) atomicOr(err, kErrTimeout);
      if (!ok) mbar_wait(&s_bar[0], 0, kWaitPolls);
      cp_async_wait_all();
      return;
    }
    // ---- kinetic pass: st <- d2 = (T - 1) s
    kinetic_pass<NR>(st, rows, s_kd, s_tw);
  } else {
    __syncthreads();
  }

  // ---- R-space pass, CH radial points at a time; thread rows row0 + i*rstep
  const int nterms = s_nterms;
  const float theta = (float)sp.theta;
  const float cfix = md.ncorr[m];  // rounding feedback of the previous step
  float a_hi[7] = {0, 0, 0, 0, 0, 0, 0}, a_lo[7] = {0, 0, 0, 0, 0, 0, 0};
  float rnd = 0.f;
  const int nchunks = NR / CH;
  for (int ck = 0; ck < nchunks; ++ck) {
    const int r0 = ck * CH, r = r0 + rl, b = ck & 1;
    float2* bU = bC + b * cbuf;
    const float2* bD = bU + rows * CH;              // streaming form: d2 of the chunk
    const float2* bV = bD + nd * CH;                // e^{-iV dtau} - 1
    const float2* bH = bV + 2 * (J + 1) * CH;       // e^{-iV dtau/2}
    const float2* bM = bH + 2 * (J + 1) * CH;
    // this chunk's copies (issued one chunk earlier) are complete and
    // visible; the other buffer is free since the previous chunk's barriers
    cp_async_wait_all();
    __syncthreads();
    if (ck + 1 < nchunks) issue_chunk(r0 + CH, b ^ 1);
    // eta = D^dagger V^{1/2} u (rotated frame) into bZ (no coupling work when E' = 0)
    float2 sacc[MAXR];
#pragma unroll
    for (int i = 0; i < MAXR; ++i) sacc[i] = make_float2(0.f, 0.f);
    if (nterms > 0) {
#pragma unroll
      for (int i = 0; i < MAXR; ++i) {
        const int row = row0 + i * rstep;
        if (row < rows) {
          const int2 ri = s_rinfo[row];
          const float2 u = (FUSED ? st[row * NRP + r] : bD[row * CH + rl]) + bU[row * CH + rl];
          bZ[row * CH + rl] = cmul(s_ph[ri.y], cmul(bH[ri.x + rl], u));
        }
      }
      __syncthreads();
    }
    float2* in = bZ;
    float2* out = bY;
    for (int n = 1; n <= nterms; ++n) {
      const float cn = theta / (float)n;
#pragma unroll
      for (int i = 0; i < MAXR; ++i) {
        const int row = row0 + i * rstep;
        if (row < rows) {
          const int sf = row >= nrot, c = row - sf * nrot;
          const float2* src = in + (1 - sf) * nrot * CH + rl;
          const int2* pr = s_prog + c * kMaxCoupl;
          float ax = 0.f, ay = 0.f;
#pragma unroll
          for (int e = 0; e < kMaxCoupl; ++e) {  // unused slots carry a zero coefficient
            const int2 q = pr[e];
            const float cf = __int_as_float(q.y);
            const float2 v = src[q.x];
            ax = fmaf(cf, v.x, ax);
            ay = fmaf(cf, v.y, ay);
          }
          const float2 o = make_float2(-cn * ay, cn * ax);  // i (theta/n) (M_r in)
          out[row * CH + rl] = o;
          sacc[i].x += o.x;
          sacc[i].y += o.y;
        }
      }
      __syncthreads();
      float2* tmp = in;
      in = out;
      out = tmp;
    }
    // d1 = (V - 1) u + V^{1/2} D S_r ; mask ; s' = s + (d2 + d1) + cfix s
    const float mk = bM[rl].x;
    float agf = 0.f, aef = 0.f;
#pragma unroll
    for (int i = 0; i < MAXR; ++i) {
      const int row = row0 + i * rstep;
      if (row < rows) {
        const int2 ri = s_rinfo[row];
        const int sf = row >= nrot;
        const float2 sv = bU[row * CH + rl];
        const float2 d2 = FUSED ? st[row * NRP + r] : bD[row * CH + rl];
        const float2 u = sv + d2;
        const float2 ph = s_ph[ri.y];
        const float2 vd = bV[ri.x + rl];
        const float2 corr = cmul(bH[ri.x + rl], cmul(make_float2(ph.x, -ph.y), sacc[i]));
        float2 d1 = make_float2(fmaf(u.x, vd.x, fmaf(-u.y, vd.y, corr.x)), fmaf(u.x, vd.y, fmaf(u.y, vd.x, corr.y)));
        if (mk < 1.f) {
          const float px = u.x + d1.x, py = u.y + d1.y;
          d1.x = fmaf(mk - 1.f, u.x, mk * d1.x);
          d1.y = fmaf(mk - 1.f, u.y, mk * d1.y);
          const float qx = u.x + d1.x, qy = u.y + d1.y;
          const float dd = fmaf(px, px, py * py) - fmaf(qx, qx, qy * qy);
          if (sf == 0) agf += dd; else aef += dd;
        }
        const float2 sn = round_update(sv, d2 + d1, cfix, rnd);
        gs[(long long)row * NR + r] = sn;
        bY[row * CH + rl] = sn;
        const float b2 = fmaf(sn.x, sn.x, sn.y * sn.y);
        if (sf == 0) acc2(a_hi[0], a_lo[0], b2);  // compensated from the first term on
        else acc2(a_hi[1], a_lo[1], b2);
      }
    }
    acc2(a_hi[2], a_lo[2], agf);
    acc2(a_hi[3], a_lo[3], aef);
    __syncthreads();
    // dipole in the molecule frame: sum_c conj(g_c) (A e)_c for A = Z, S+, S-
    {
      float2 accP = make_float2(0.f, 0.f), accM = accP, accZ = accP;
      for (int c = row0; c < nrot; c += rstep) {
        const float2 gc = bY[c * CH + rl];
        const float2* ee = bY + nrot * CH + rl;
        const int2* pr = s_dipp + c * kMaxCoupl;
        float2 w3[3];
#pragma unroll
        for (int kk = 0; kk < 3; ++kk) {  // slots 0-1 Z, 2-3 S+, 4-5 S- (unused: zero coefficient)
          const int2 q0 = pr[2 * kk], q1 = pr[2 * kk + 1];
          const float c0 = __int_as_float(q0.y), c1 = __int_as_float(q1.y);
          const float2 e0 = ee[q0.x], e1 = ee[q1.x];
          w3[kk] = make_float2(fmaf(c0, e0.x, c1 * e1.x), fmaf(c0, e0.y, c1 * e1.y));
        }
        // conj(gc) * w
        accZ.x += fmaf(gc.x, w3[0].x, gc.y * w3[0].y);
        accZ.y += fmaf(gc.x, w3[0].y, -gc.y * w3[0].x);
        accP.x += fmaf(gc.x, w3[1].x, gc.y * w3[1].y);
        accP.y += fmaf(gc.x, w3[1].y, -gc.y * w3[1].x);
        accM.x += fmaf(gc.x, w3[2].x, gc.y * w3[2].y);
        accM.y += fmaf(gc.x, w3[2].y, -gc.y * w3[2].x);
      }
      acc2(a_hi[4], a_lo[4], accP.x + accM.x);
      acc2(a_hi[5], a_lo[5], accP.y - accM.y);
      acc2(a_hi[6], a_lo[6], 2.f * accZ.x);
    }
    __syncthreads();
  }
  // ---- block reduction (compensated FP32; FP64 only for the final sums)
  {
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      float hi = q < 7 ? a_hi[q] : rnd, lo = q < 7 ? a_lo[q] : 0.f;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const float h2 = __shfl_xor_sync(0xffffffffu, hi, o);
        const float l2 = __shfl_xor_sync(0xffffffffu, lo, o);
        acc2(hi, lo, h2);
        lo += l2;
      }
      if (lane == 0) s_red[w][q] = make_float2(hi, lo);
    }
    __syncthreads();
    if (t < 8) {  // one quantity per thread, compensated over the warps
      float hi = 0.f, lo = 0.f;
      for (int ww = 0; ww < NW; ++ww) {
        acc2(hi, lo, s_red[ww][t].x);
        lo += s_red[ww][t].y;
      }
      s_fin[t] = hi + lo;  // FP32 sum; its rounding is 6e-8 relative
      s_fin_lo[t] = lo - (s_fin[t] - hi);
    }
    __syncthreads();
    if (t < 3) {  // lab dipole component t: mu = O mu', mu' = d dR (Re(S+ + S-), Im(S+ - S-), 2 Re Z)
      const float sc = (float)sp.dipole * sp.dR;
      const float lab = sc * (s_rot[3 * t] * s_fin[4] + s_rot[3 * t + 1] * s_fin[5] + s_rot[3 * t + 2] * s_fin[6]);
      const double nl = (double)lab;
      md.dmu[3 * (long long)m + t] = nl - s_mu[t];
      md.mu[3 * (long long)m + t] = nl;
    } else if (t < 5) {  // populations P_g, P_e
      const double P = ((double)s_fin[t - 3] + (double)s_fin_lo[t - 3]) * (double)sp.dR;
      md.pop[2 * (long long)m + (t - 3)] = P;
      if (!isfinite(P)) atomicOr(err, kErrNonFinite);
    } else if (t < 7) {  // absorbed norm, cumulative
      md.absorbed[2 * (long long)m + (t - 5)] =
          s_abs[t - 5] + ((double)s_fin[t - 3] + (double)s_fin_lo[t - 3]) * (double)sp.dR;
    } else if (t == 7) {  // rounding feedback for the next step
      md.ncorr[m] = rounding_feedback(s_fin[7], s_fin[0] + s_fin[1]);
    }
  }
}


// ----------------------------------------------------------------------------
// R-space pass of the streaming form, tiled: one CTA per molecule at a time,
// TILE = 32 or 16 radial points per tile, every row of the state.  The rows
// (surface, channel) are spread over the warps and stay in registers for a
// tile: s and d2 = (T - 1) s arrive by 2-D tensor copies and the coupling
// series exchanges values between rows through two term buffers in shared
// memory.
//
// Neighbour structure: the angular couplings of channel (j, m) reach the
// channels (j + 1, m - 1 .. m + 1) and (j - 1, m - 1 .. m + 1), two runs of
// three consecutive channels (c + 2j + 1 .. c + 2j + 3 and c - 2j - 1 ..
// c - 2j + 1, c = j^2 + j + m).  A row therefore needs two base offsets and
// six coefficients: for the coupling E_perp X + E'_z Z in the turned frame
// (X = (S+ + S-)/2) and for the dipole (Z, S+, S-).  Coefficients of channels
// outside the basis are zero and their reads land on finite data: kTriGuard
// zero rows precede each buffer, and a missing run points at them.
// ----------------------------------------------------------------------------
// The angular tables of every translation unit's copy.
cudaError_t upload_triplet_tables(const CouplEntry* dip) {
  cudaError_t e = upload_triplet_tables_local(dip);
  if (e == cudaSuccess) e = upload_triplet_tables_tile(dip);
  if (e != cudaSuccess) return e;
  return upload_triplet_tables_pair(dip);
}

// Diagnostic of the bounded wait: one CTA waits on a barrier that nothing
// completes, gives up after `tries` tries of up to 10 us, and records the
// timeout as the molecular kernels do.
__global__ void wait_timeout_probe_kernel(int tries, int* flag) {
  __shared__ __align__(8) unsigned long long bar[1];
  if (threadIdx.x == 0) {
    mbar_init(&bar[0], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  const bool ok = mbar_wait_sleep(&bar[0], 0, tries, 10000u);
  if (!__syncthreads_and(ok) && threadIdx.x == 0) atomicOr(flag, kErrTimeout);
}

// Latches a host-detected launch failure into the error word.
__global__ void flag_error_kernel(int* err, int code) { atomicOr(err, code); }

cudaError_t launch_wait_timeout_probe(int tries, int* flag, cudaStream_t s) {
  wait_timeout_probe_kernel<<<1, 32, 0, s>>>(tries, flag);
  return cudaGetLastError();
}

// ----------------------------------------------------------------------------
// R-space pass of the streaming form, point-resident layout (J <= 4): one CTA
// per molecule, one thread per (radial point, surface).  A thread holds the
// channel vector of its surface at its point in registers, so the angular
// couplings become register arithmetic with indices fixed at compile time;
// the coupling series (sigma_x swaps the surfaces) and the dipole only
// exchange the other surface's vector, through one shared buffer.
// ----------------------------------------------------------------------------
template <int I, int N, class F>
__device__ __forceinline__ void static_for(F&& f) {
  if constexpr (I < N) {
    f(std::integral_constant<int, I>());
    static_for<I + 1, N>(f);
  }
}
constexpr int ch_j(int c) { return c < 1 ? 0 : (c < 4 ? 1 : (c < 9 ? 2 : (c < 16 ? 3 : (c < 25 ? 4 : -1)))); }
__host__ __device__ constexpr int j_of_c(int c) { return ch_j(c); }
constexpr int ch_m(int c) { return c - ch_j(c) * ch_j(c) - ch_j(c); }
// channel of (j, m), or -1 outside the basis of size J
constexpr int ch_of(int j, int m, int J) { return (j < 0 || j > J || m < -j || m > j) ? -1 : j * j + j + m; }

// ---- angular coefficients as compile-time constants ------------------------
// square root by Newton's iteration in double precision (x >= 0)
constexpr double c_sqrt(double x) {
  if (x <= 0.0) return 0.0;
  double r = x < 1.0 ? 1.0 : x;
  for (int i = 0; i < 64; ++i) r = 0.5 * (r + x / r);
  return r;
}
constexpr bool ch_valid(int j, int m) { return j >= 0 && m >= -j && m <= j; }
// <j+1, m|cos t|j, m>, -<j+1, m+1|sin t e^{i p}|j, m> and <j-1, m+1|sin t e^{i p}|j, m>
// in the Condon-Shortley phase convention
constexpr double c_ang_a(int j, int m) {
  return c_sqrt(((j + 1.0) * (j + 1) - (double)m * m) / ((2.0 * j + 1) * (2.0 * j + 3)));
}
constexpr double c_ang_b(int j, int m) {
  return -c_sqrt((j + m + 1.0) * (j + m + 2) / ((2.0 * j + 1) * (2.0 * j + 3)));
}
constexpr double c_ang_c(int j, int m) {
  return c_sqrt((j - m) * (j - m - 1.0) / ((2.0 * j - 1) * (2.0 * j + 1)));
}
// Row (j, m) of Z, S+ = sin t e^{ip} and S- = sin t e^{-ip} on the runs (j + 1, .) and (j - 1, .):
// Z from (j +- 1, m), S+ from (j +- 1, m - 1), S- from (j +- 1, m + 1).
constexpr float c_zu(int j, int m) { return (float)c_ang_a(j, m); }
constexpr float c_zd(int j, int m) { return ch_valid(j - 1, m) ? (float)c_ang_a(j - 1, m) : 0.f; }
constexpr float c_pu(int j, int m) { return ch_valid(j + 1, m - 1) ? (float)c_ang_c(j + 1, m - 1) : 0.f; }
constexpr float c_pd(int j, int m) { return ch_valid(j - 1, m - 1) ? (float)c_ang_b(j - 1, m - 1) : 0.f; }
constexpr float c_mu(int j, int m) { return (float)c_ang_b(j, m); }
constexpr float c_md(int j, int m) { return j >= 1 ? (float)c_ang_c(j, m) : 0.f; }

// Per molecule of a streaming species: the local field in the molecule frame
// scaled by theta, (theta E'_z, theta E'_x / 2, theta E'_y / 2), and the
// number of coupling-series terms (coupling_terms).
__global__ void mol_field_kernel(SpeciesDev sp, MolDev md, Grid g, int prescribed, int* err) {
  const int lm = blockIdx.x * blockDim.x + threadIdx.x;
  if (lm >= sp.nmol) return;
  const int m = sp.mol[lm];
  float E[3];
  lab_field(md, g, prescribed, m, E, err);
  const float* O = md.rot + 9 * (long long)m;  // molecule -> lab, row-major
  const float inv_fau = 1.0f / 5.14220674763e11f;
  float Ep[3];
#pragma unroll
  for (int i = 0; i < 3; ++i) Ep[i] = (O[i] * E[0] + O[3 + i] * E[1] + O[6 + i] * E[2]) * inv_fau;
  const float th = (float)sp.theta;
  const float x = th * sqrtf(Ep[0] * Ep[0] + Ep[1] * Ep[1] + Ep[2] * Ep[2]);
  if (!isfinite(x)) atomicOr(err, kErrNonFinite);  // a non-finite local field
  const int nt = coupling_terms(x);
  if (nt >= 24 || x > 4.f) atomicOr(err, kErrCouplingSeries);
  sp.fld[lm] = make_float4(th * Ep[2], 0.5f * th * Ep[0], 0.5f * th * Ep[1], __int_as_float(nt));
}

// Row layout of a molecule's state.  Full: both surfaces carry every channel
// c = j^2 + j + m, c < (J+1)^2, in channel order.  Parity-reduced: starting
// from j = 0 on the ground surface, the couplings (j -> j +- 1, surfaces
// swapped) only ever populate (ground, even j) and (excited, odd j), so only
// those rows are stored: ground rows are the even-j channels, excited rows
// the odd-j channels, each in channel order.
template <int J, bool PAR>
struct Rows {
  static constexpr int NROT = (J + 1) * (J + 1);
  static constexpr int count(int q) {  // channels of j parity q up to J
    int n = 0;
    for (int j = q; j <= J; j += 2) n += 2 * j + 1;
    return n;
  }
  static constexpr int NG = PAR ? count(0) : NROT;  // ground rows
  static constexpr int NE = PAR ? count(1) : NROT;  // excited rows
  static constexpr int ROWS = NG + NE;
  static constexpr int N(int sf) { return sf ? NE : NG; }
  static constexpr int base(int sf) { return sf ? NG : 0; }  // first row of surface sf
  // channel stored in row r of surface sf
  static constexpr int chan(int sf, int r) {
    if (!PAR) return r;
    for (int j = sf; j <= J; j += 2) {
      if (r < 2 * j + 1) return j * j + r;
      r -= 2 * j + 1;
    }
    return -1;
  }
  // row of surface sf holding channel c (-1: c outside the basis or not stored)
  static constexpr int row(int sf, int c) {
    if (c < 0) return -1;
    if (!PAR) return c;
    const int j = ch_j(c);
    if ((j & 1) != sf) return -1;
    int r = 0;
    for (int jj = sf; jj < j; jj += 2) r += 2 * jj + 1;
    return r + (c - j * j);
  }
};

// i (theta/n) (M in) for row R of surface SF, M = E'_z Z + (E'_x - i E'_y)/2 S+
// + (E'_x + i E'_y)/2 S- (the molecule-frame coupling), `in` the other
// surface's rows; f = (theta E'_z, theta E'_x/2, theta E'_y/2)
template <int J, bool PAR, int SF, int R, class V>
__device__ __forceinline__ float2 coupling_row(const V& in, float fz, float fx, float fy, float cn) {
  using L = Rows<J, PAR>;
  constexpr int C = L::chan(SF, R), j = ch_j(C), mm = ch_m(C);
  float2 az = make_float2(0.f, 0.f), ap = az, am = az;
  auto mac = [&](float2& a, float cf, auto ni) {
    constexpr int q = decltype(ni)::value;
    if constexpr (q >= 0) {
      a.x = fmaf(cf, in[q].x, a.x);
      a.y = fmaf(cf, in[q].y, a.y);
    }
  };
  if constexpr (j < J) {
    mac(az, c_zu(j, mm), std::integral_constant<int, L::row(1 - SF, ch_of(j + 1, mm, J))>());
    mac(ap, c_pu(j, mm), std::integral_constant<int, L::row(1 - SF, ch_of(j + 1, mm - 1, J))>());
    mac(am, c_mu(j, mm), std::integral_constant<int, L::row(1 - SF, ch_of(j + 1, mm + 1, J))>());
  }
  if constexpr (j > 0) {
    mac(az, c_zd(j, mm), std::integral_constant<int, c_zd(j, mm) != 0.f ? L::row(1 - SF, ch_of(j - 1, mm, J)) : -1>());
    mac(ap, c_pd(j, mm),
        std::integral_constant<int, c_pd(j, mm) != 0.f ? L::row(1 - SF, ch_of(j - 1, mm - 1, J)) : -1>());
    mac(am, c_md(j, mm),
        std::integral_constant<int, c_md(j, mm) != 0.f ? L::row(1 - SF, ch_of(j - 1, mm + 1, J)) : -1>());
  }
  // a = fz Z-part + fx (S+ + S-) - i fy (S+ - S-)
  const float bx = ap.x + am.x, by = ap.y + am.y, cx = ap.x - am.x, cy = ap.y - am.y;
  const float ax = fmaf(fz, az.x, fmaf(fx, bx, fy * cy));
  const float ay = fmaf(fz, az.y, fmaf(fx, by, -fy * cx));
  return make_float2(-cn * ay, cn * ax);
}

// Dipole sums of ground rows [R0, R1): sum_c conj(g_c) (A e)_c for A = S+, S-,
// Z (g the ground rows, e the excited rows at one radial point)
template <int J, bool PAR, int R, class V, class W>
__device__ __forceinline__ void dipole_row(const V& gv, const W& ev, float2& accP, float2& accM, float2& accZ) {
  using L = Rows<J, PAR>;
  constexpr int C = L::chan(0, R), j = ch_j(C), mm = ch_m(C);
  float2 wP = make_float2(0.f, 0.f), wZ = wP, wM = wP;
  auto mac = [&](float2& a, float cf, auto ni) {
    constexpr int q = decltype(ni)::value;
    if constexpr (q >= 0) {
      a.x = fmaf(cf, ev[q].x, a.x);
      a.y = fmaf(cf, ev[q].y, a.y);
    }
  };
  if constexpr (j < J) {
    mac(wZ, c_zu(j, mm), std::integral_constant<int, L::row(1, ch_of(j + 1, mm, J))>());
    mac(wP, c_pu(j, mm), std::integral_constant<int, L::row(1, ch_of(j + 1, mm - 1, J))>());
    mac(wM, c_mu(j, mm), std::integral_constant<int, L::row(1, ch_of(j + 1, mm + 1, J))>());
  }
  if constexpr (j > 0) {
    mac(wZ, c_zd(j, mm), std::integral_constant<int, c_zd(j, mm) != 0.f ? L::row(1, ch_of(j - 1, mm, J)) : -1>());
    mac(wP, c_pd(j, mm), std::integral_constant<int, c_pd(j, mm) != 0.f ? L::row(1, ch_of(j - 1, mm - 1, J)) : -1>());
    mac(wM, c_md(j, mm), std::integral_constant<int, c_md(j, mm) != 0.f ? L::row(1, ch_of(j - 1, mm + 1, J)) : -1>());
  }
  const float2 gc = gv[R];
  accZ.x += fmaf(gc.x, wZ.x, gc.y * wZ.y);
  accZ.y += fmaf(gc.x, wZ.y, -gc.y * wZ.x);
  accP.x += fmaf(gc.x, wP.x, gc.y * wP.y);
  accP.y += fmaf(gc.x, wP.y, -gc.y * wP.x);
  accM.x += fmaf(gc.x, wM.x, gc.y * wM.y);
  accM.y += fmaf(gc.x, wM.y, -gc.y * wM.x);
}
template <int J, bool PAR, int R0, int R1, class V, class W>
__device__ __forceinline__ void dipole_rows(const V& gv, const W& ev, float2& accP, float2& accM, float2& accZ) {
  if constexpr (R0 < R1) {
    dipole_row<J, PAR, R0>(gv, ev, accP, accM, accZ);
    dipole_rows<J, PAR, R0 + 1, R1>(gv, ev, accP, accM, accZ);
  }
}

// Point-resident R-space pass (and, FUSED, the kinetic pass): one CTA of 2 N_r
// threads per molecule, thread = (radial point, surface); PAR: parity-reduced
// rows.  FUSED (N_r = 128): the state is staged once into D and turned in
// place into d2 = (T - 1) s by the shared-memory FFT, while a second copy of
// s (an L2 hit) fills X.  Otherwise d2 comes from the kinetic kernel's
// scratch.  Every CTA barrier sits in code all threads run; the per-surface
// work between them is compiled once per surface (row counts differ when
// PAR).
template <int J, int NR, bool FUSED, bool PAR, bool DIPR = false>
__global__ void __launch_bounds__(2 * NR, NR <= 64 ? 4 : (NR <= 128 ? (PAR ? 3 : 2) : 1))
    mol_rpoint_kernel(SpeciesDev sp, MolDev md, int* err) {
  using L = Rows<J, PAR>;
  constexpr int ROWS = L::ROWS, NG = L::NG, NT = 2 * NR, NW = NT / 32;
  constexpr int RMAX = L::NG > L::NE ? L::NG : L::NE;
  constexpr unsigned kStateBytes = (unsigned)ROWS * NR * sizeof(float2);  // one molecule's state
  static_assert(!FUSED || NT == FFTShape<NR>::THREADS, "the fused form runs the FFT with every thread");
  extern __shared__ __align__(16) float4 smem4[];
  float2* X = reinterpret_cast<float2*>(smem4);  // [ROWS][NR]: s, then eta and the series terms, then s'
  float2* D = X + ROWS * NR;                     // [ROWS][NR]: d2
  float2* s_tw = D + ROWS * NR;                  // fused: [N2][N1] FFT twiddles
  float2* s_kd = s_tw + NR;                      // fused: [NR] kinetic phase deltas
  __shared__ __align__(8) unsigned long long s_bar[2];
  __shared__ float s_rot[9];
  __shared__ double s_mu[3], s_abs[2];
  __shared__ float s_red[NW][10];
  __shared__ float s_fin[8], s_fin_lo[2];

  const int t = threadIdx.x, lane = t & 31, w = t >> 5;
  const int sf = t >= NR, p = t - sf * NR;  // surface (warp-uniform) and radial point
  const int lm = blockIdx.x;
  const int m = sp.mol[lm];
  const long long mol0 = (long long)lm * ROWS * NR;  // first element of this molecule
  const int own0 = sf ? NG : 0, oth0 = sf ? 0 : NG;   // first rows of this and the other surface
  float2* gs = sp.psi + mol0 + (long long)own0 * NR + p;
  float2* Xo = X + own0 * NR + p;        // own rows
  const float2* Xt = X + oth0 * NR + p;  // the other surface's rows
  const float2* Do = D + own0 * NR + p;
  const float2* vdp = sp.vdelta + sf * (J + 1) * NR + p;
  const float2* vhp = sp.vhalf + sf * (J + 1) * NR + p;

  // the molecule's state (and d2), one bulk copy each (contiguous in global memory)
  if (t == 0) {
    mbar_init(&s_bar[0], 1);
    mbar_init(&s_bar[1], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    if (FUSED) {
      mbar_expect_tx(&s_bar[0], kStateBytes);
      bulk_g2s(D, sp.psi + mol0, kStateBytes, &s_bar[0]);
    } else {
      mbar_expect_tx(&s_bar[0], 2 * kStateBytes);
      bulk_g2s(X, sp.psi + mol0, kStateBytes, &s_bar[0]);
      bulk_g2s(D, sp.d2 + mol0, kStateBytes, &s_bar[0]);
    }
  }
  if (FUSED) {
    for (int q = t; q < NR; q += NT) {
      s_tw[q] = __ldg(&sp.twiddle[q]);
      s_kd[q] = __ldg(&sp.kdelta[q]);
    }
  }
  if (t >= 32 && t < 41) s_rot[t - 32] = md.rot[9 * (long long)m + (t - 32)];
  else if (t >= 64 && t < 67) s_mu[t - 64] = md.mu[3 * (long long)m + (t - 64)];
  else if (t >= 67 && t < 69) s_abs[t - 67] = md.absorbed[2 * (long long)m + (t - 67)];
  // theta E' of the molecule, times d(R) / max|d| at this thread's point
  // (1 for a constant dipole)
  float4 f = __ldg(&sp.fld[lm]);
  if constexpr (DIPR) {
    const float dw = __ldg(&sp.dipw[p]);
    f.x *= dw;
    f.y *= dw;
    f.z *= dw;
  }
  const int nterms = __float_as_int(f.w);
  const float mk = sp.maskw[p].x;
  const float cfix = md.ncorr[m];  // rounding feedback of the previous step
  float2 vh[J + 1], vd[J + 1];
#pragma unroll
  for (int j = 0; j <= J; ++j) {
    vd[j] = __ldg(vdp + j * NR);
    vh[j] = __ldg(vhp + j * NR);
  }
  __syncthreads();  // the barrier is initialised
  auto wait_all = [&](int id) -> bool {
    const bool ok = mbar_wait_sleep(&s_bar[id], 0);
    if (__syncthreads_and(ok)) return true;
    if (t == 0) atomicOr(err, kErrTimeout);
    if (!ok) mbar_wait_sleep(&s_bar[id], 0);
    return false;
  };
  if (!wait_all(0)) return;
  if (FUSED) {
    if (t == 0) {  // s again into X (the lines were just read), while the FFT runs on D
      mbar_expect_tx(&s_bar[1], kStateBytes);
      bulk_g2s(X, sp.psi + mol0, kStateBytes, &s_bar[1]);
    }
    kinetic_pass<NR>(D, ROWS, s_kd, s_tw);  // D <- d2 = (T - 1) s
    if (!wait_all(1)) return;
  }
  // per-surface work: both surfaces share one row list in the full layout
  auto per_surface = [&](auto&& fn) {
    if constexpr (PAR) {
      if (sf == 0) fn(std::integral_constant<int, 0>());
      else fn(std::integral_constant<int, 1>());
    } else {
      fn(std::integral_constant<int, 0>());
    }
  };
  // ---- eta = V^{1/2} u, u = s + d2, over this thread's own rows of the state
  auto eta = [&](auto sfc) {
    constexpr int SF = decltype(sfc)::value;
    static_for<0, L::N(SF)>([&](auto ri) {
      constexpr int r = decltype(ri)::value, j = ch_j(L::chan(SF, r));
      Xo[r * NR] = cmul(vh[j], Xo[r * NR] + Do[r * NR]);
    });
  };
  if (nterms > 0) per_surface(eta);
  __syncthreads();
  // ---- coupling series: S = sum_n (i theta M sigma_x)^n eta / n!
  float2 sacc[RMAX], in[RMAX];
#pragma unroll
  for (int r = 0; r < RMAX; ++r) sacc[r] = make_float2(0.f, 0.f);
  auto term = [&](auto sfc, float cn, bool store) {
    constexpr int SF = decltype(sfc)::value;
    static_for<0, L::N(SF)>([&](auto ri) {
      constexpr int r = decltype(ri)::value;
      const float2 o = coupling_row<J, PAR, SF, r>(in, f.x, f.y, f.z, cn);
      sacc[r].x += o.x;
      sacc[r].y += o.y;
      if (store) Xo[r * NR] = o;
    });
  };
  const int n_oth = PAR ? (sf ? L::NG : L::NE) : L::NROT;
  for (int n = 1; n <= nterms; ++n) {
#pragma unroll
    for (int r = 0; r < RMAX; ++r)
      if (r < n_oth) in[r] = Xt[r * NR];
    __syncthreads();  // every thread has its input: the buffer may be overwritten
    const float cn = 1.f / (float)n;
    const bool store = n < nterms;
    per_surface([&](auto sfc) { term(sfc, cn, store); });
    if (store) __syncthreads();
  }
  // ---- d1 = (V - 1) u + V^{1/2} S ; mask ; s' = s + (d2 + d1) + cfix s
  float sn2 = 0.f, sn2_lo = 0.f, absd = 0.f, rnd = 0.f;  // |s'|^2 compensated from the first term on
  auto update = [&](auto sfc) {
    constexpr int SF = decltype(sfc)::value, NO = L::N(SF);
    // s again (from L2), in two batches each requested in full first; d2 from shared memory
    constexpr int NB = NO > 1 ? (NO + 1) / 2 : 1;
    float2 sb[NB];
    auto fetch = [&](int r0) {
#pragma unroll
      for (int k = 0; k < NB; ++k)
        if (r0 + k < NO) sb[k] = __ldcs(gs + (r0 + k) * NR);
    };
    fetch(0);
    static_for<0, NO>([&](auto ri) {
      constexpr int r = decltype(ri)::value, j = ch_j(L::chan(SF, r));
      if constexpr (r == NB) fetch(NB);
      const float2 sv = sb[r % NB], dv = Do[r * NR];
      const float2 u = sv + dv;
      float2 d1 = cmul(vd[j], u);
      if (nterms > 0) d1 = d1 + cmul(vh[j], sacc[r]);
      if (mk < 1.f) {
        const float px = u.x + d1.x, py = u.y + d1.y;
        d1.x = fmaf(mk - 1.f, u.x, mk * d1.x);
        d1.y = fmaf(mk - 1.f, u.y, mk * d1.y);
        absd += (1.f - mk * mk) * fmaf(px, px, py * py);
      }
      const float2 s1 = round_update(sv, dv + d1, cfix, rnd);
      __stcs(gs + r * NR, s1);
      acc2(sn2, sn2_lo, fmaf(s1.x, s1.x, s1.y * s1.y));
      sacc[r] = s1;  // the new state of this surface, kept for the dipole
      Xo[r * NR] = s1;
    });
  };
  per_surface(update);
  __syncthreads();
  // ---- dipole in the molecule frame: sum over ground rows of conj(g_c) (A e)_c
  // for A = Z, S+, S-; ground rows [0, NH) on the ground-surface threads, the
  // rest on the excited ones
  float dP = 0.f, dQ = 0.f, dZ = 0.f;
  {
    constexpr int NH = (NG + 1) / 2;
#pragma unroll
    for (int r = 0; r < RMAX; ++r)
      if (r < n_oth) in[r] = Xt[r * NR];
    float2 accP = make_float2(0.f, 0.f), accM = accP, accZ = accP;
    if (sf == 0) dipole_rows<J, PAR, 0, NH>(sacc, in, accP, accM, accZ);
    else dipole_rows<J, PAR, NH, NG>(in, sacc, accP, accM, accZ);
    dP = accP.x + accM.x;
    dQ = accP.y - accM.y;
    dZ = 2.f * accZ.x;
  }
  // ---- block reduction: populations compensated, the rest plain FP32
  {
    float v[8] = {sf ? 0.f : sn2, sf ? sn2 : 0.f, sf ? 0.f : absd, sf ? absd : 0.f, dP, dQ, dZ, rnd};
    float lo[2] = {sf ? 0.f : sn2_lo, sf ? sn2_lo : 0.f};
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
      if constexpr (!DIPR) {  // with d(R) the dipole is read from T^{1/2} s' by mol_dipole_r_kernel
        const float sc = (float)sp.dipole * sp.dR;
        const float lab = sc * (s_rot[3 * t] * s_fin[4] + s_rot[3 * t + 1] * s_fin[5] + s_rot[3 * t + 2] * s_fin[6]);
        const double nl = (double)lab;
        md.dmu[3 * (long long)m + t] = nl - s_mu[t];
        md.mu[3 * (long long)m + t] = nl;
      }
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

template <int J, int NR, bool FUSED, bool PAR, bool DIPR = false>
static void launch_rpoint_jnp(const SpeciesDev& sp, const MolDev& md, int* err, cudaStream_t s) {
  constexpr int ROWS = Rows<J, PAR>::ROWS;
  const size_t smem = (size_t)2 * ROWS * NR * sizeof(float2) + (FUSED ? 2 * NR * sizeof(float2) : 0);
  auto k = mol_rpoint_kernel<J, NR, FUSED, PAR, DIPR>;
  cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  cudaFuncSetAttribute(k, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
  k<<<sp.nmol, 2 * NR, smem, s>>>(sp, md, err);
}
template <int J, int NR, bool FUSED>
static void launch_rpoint_jn(const SpeciesDev& sp, const MolDev& md, int* err, cudaStream_t s) {
  if constexpr (NR <= 128) {  // R-dependent dipole: full state, N_r 64 or 128
    if (sp.dipw) {
      launch_rpoint_jnp<J, NR, FUSED, false, true>(sp, md, err, s);
      return;
    }
  }
  if (sp.par) launch_rpoint_jnp<J, NR, FUSED, true>(sp, md, err, s);
  else launch_rpoint_jnp<J, NR, FUSED, false>(sp, md, err, s);
}

template <int NR, bool FUSED = false>
static void launch_rpoint_n(const SpeciesDev& sp, const MolDev& md, int* err, cudaStream_t s) {
  switch (sp.jmax) {
    case 0: launch_rpoint_jn<0, NR, FUSED>(sp, md, err, s); break;
    case 1: launch_rpoint_jn<1, NR, FUSED>(sp, md, err, s); break;
    case 2: launch_rpoint_jn<2, NR, FUSED>(sp, md, err, s); break;
    case 3: launch_rpoint_jn<3, NR, FUSED>(sp, md, err, s); break;
    case 4: launch_rpoint_jn<4, NR, FUSED>(sp, md, err, s); break;
  }
}

// Dipole of a species with an R-dependent transition dipole d(R).  The
// stored state is s = T^{-1/2} psi; the populations are the same from s and
// psi (T^{1/2} is unitary per channel), and so is the dipole while d is
// constant (T commutes with d sigma_x (x) R^).  With d(R) it does not, so the
// dipole is taken from psi' = T^{1/2} s' after the step: one CTA per
// molecule stages s', turns it into psi' with the shared-memory FFT and sums
// 2 Re sum_R d(R) g^dagger A e dR for A = S+, S-, Z (threads t < N_r: one
// radial point each), then writes mu and the change over the step.
template <int J, int NR, bool PAR>
__global__ void __launch_bounds__(FFTShape<NR>::THREADS) mol_dipole_r_kernel(SpeciesDev sp, MolDev md, int* err) {
  using L = Rows<J, PAR>;
  constexpr int ROWS = L::ROWS, NG = L::NG, NE = L::NE, NT = FFTShape<NR>::THREADS, NW = NT / 32;
  constexpr unsigned kStateBytes = (unsigned)ROWS * NR * sizeof(float2);
  extern __shared__ __align__(16) float4 smem4[];
  float2* X = reinterpret_cast<float2*>(smem4);  // [ROWS][NR]: s', then psi'
  float2* s_tw = X + ROWS * NR;
  float2* s_kh = s_tw + NR;
  __shared__ __align__(8) unsigned long long s_bar[1];
  __shared__ float s_red[NW][3];
  const int t = threadIdx.x, lane = t & 31, w = t >> 5;
  const int lm = blockIdx.x;
  const int m = sp.mol[lm];
  if (t == 0) {
    mbar_init(&s_bar[0], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    mbar_expect_tx(&s_bar[0], kStateBytes);
    bulk_g2s(X, sp.psi + (long long)lm * ROWS * NR, kStateBytes, &s_bar[0]);
  }
  for (int q = t; q < NR; q += NT) {
    s_tw[q] = __ldg(&sp.twiddle[q]);
    s_kh[q] = __ldg(&sp.khalf[q]);
  }
  __syncthreads();
  const bool ok = mbar_wait_sleep(&s_bar[0], 0);
  if (!__syncthreads_and(ok)) {
    if (t == 0) atomicOr(err, kErrTimeout);
    if (!ok) mbar_wait_sleep(&s_bar[0], 0);
    return;
  }
  kinetic_pass<NR>(X, ROWS, s_kh, s_tw);  // psi' = T^{1/2} s'
  float dP = 0.f, dQ = 0.f, dZ = 0.f;
  if (t < NR) {
    float2 gv[NG], ev[NE > 0 ? NE : 1];  // J = 0, parity-reduced: no excited row
#pragma unroll
    for (int r = 0; r < NG; ++r) gv[r] = X[r * NR + t];
#pragma unroll
    for (int r = 0; r < NE; ++r) ev[r] = X[(NG + r) * NR + t];
    float2 accP = make_float2(0.f, 0.f), accM = accP, accZ = accP;
    dipole_rows<J, PAR, 0, NG>(gv, ev, accP, accM, accZ);
    const float d = (float)sp.dipole * __ldg(&sp.dipw[t]);
    dP = d * (accP.x + accM.x);
    dQ = d * (accP.y - accM.y);
    dZ = d * 2.f * accZ.x;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    dP += __shfl_xor_sync(0xffffffffu, dP, o);
    dQ += __shfl_xor_sync(0xffffffffu, dQ, o);
    dZ += __shfl_xor_sync(0xffffffffu, dZ, o);
  }
  if (lane == 0) {
    s_red[w][0] = dP;
    s_red[w][1] = dQ;
    s_red[w][2] = dZ;
  }
  __syncthreads();
  if (t < 3) {
    float v[3] = {0.f, 0.f, 0.f};
    for (int ww = 0; ww < NW; ++ww)
      for (int k = 0; k < 3; ++k) v[k] += s_red[ww][k];
    const float* O = md.rot + 9 * (long long)m;  // molecule -> lab, row-major
    const double lab = (double)(sp.dR * (O[3 * t] * v[0] + O[3 * t + 1] * v[1] + O[3 * t + 2] * v[2]));
    md.dmu[3 * (long long)m + t] = lab - md.mu[3 * (long long)m + t];
    md.mu[3 * (long long)m + t] = lab;
  }
}

template <int J, int NR>
static void launch_dipole_r_jn(const SpeciesDev& sp, const MolDev& md, int* err, cudaStream_t s) {
  auto run = [&](auto k, int rows) {
    const size_t smem = ((size_t)rows * NR + 2 * NR) * sizeof(float2);
    cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k<<<sp.nmol, FFTShape<NR>::THREADS, smem, s>>>(sp, md, err);
  };
  run(mol_dipole_r_kernel<J, NR, false>, Rows<J, false>::ROWS);  // d(R): full state only
}

template <int NR>
static void launch_dipole_r(const SpeciesDev& sp, const MolDev& md, int* err, cudaStream_t s) {
  switch (sp.jmax) {
    case 0: launch_dipole_r_jn<0, NR>(sp, md, err, s); break;
    case 1: launch_dipole_r_jn<1, NR>(sp, md, err, s); break;
    case 2: launch_dipole_r_jn<2, NR>(sp, md, err, s); break;
    case 3: launch_dipole_r_jn<3, NR>(sp, md, err, s); break;
    case 4: launch_dipole_r_jn<4, NR>(sp, md, err, s); break;
  }
}

// The point-resident kernel runs a species' R-space pass (and, fused, its
// kinetic pass) where it applies (J <= 4; fused only at N_r = 128) unless the
// species' plan names another kernel.
static bool use_point(const SpeciesDev& sp) {
  if (sp.jmax > 4 || (sp.path == MS_MOL_FUSED && sp.nr != 128)) return false;
  return sp.kern == MS_KERN_DEFAULT || sp.kern == MS_KERN_POINT;
}
static bool rspace_ok(int nr, int jmax);
// The tiled kernel runs a streaming species' R-space pass where the point-
// resident one does not and it applies, unless the plan names another kernel.
static bool pair_ok(int nr, int jmax) { return (nr == 64 || nr == 128 || nr == 256) && jmax <= 16; }
// The two-points-a-thread tiled kernel runs a streaming species' R-space pass
// where the plan names it, and by the static rule from J = 5 on (for the
// parity-reduced state it is the only kernel from J = 5 on).
static bool use_pair(const SpeciesDev& sp) {
  if (sp.path != MS_MOL_STREAMING || sp.dipw || !pair_ok(sp.nr, sp.jmax)) return false;
  if (sp.par) return sp.jmax >= 5;
  return sp.kern == MS_KERN_PAIR || (sp.kern == MS_KERN_DEFAULT && sp.jmax >= 5);
}
static bool use_tile(const SpeciesDev& sp) {
  if (sp.path != MS_MOL_STREAMING || use_point(sp) || use_pair(sp) || !rspace_ok(sp.nr, sp.jmax)) return false;
  return sp.kern == MS_KERN_DEFAULT || sp.kern == MS_KERN_TILE;
}
// its tile width: 8 points from J = 9 on; else the plan's, or 8 points from
// J = 5 on (the nanohole pass 113.7 against 118.3 ms at 16) and 32 below;
// parity-reduced rows: 16 points to J = 8 (at 8 a CTA would hold two warps)
static int pair_tile(const SpeciesDev& sp) {
  if (sp.jmax >= 9) return 8;
  if (sp.par) return 16;
  if (sp.ch == 8 || sp.ch == 16 || sp.ch == 32) return sp.ch;
  return sp.jmax >= 5 ? 8 : 32;
}
}  // namespace ms

// ----------------------------------------------------------------------------
// Eq. 8 readout: psi = T^{1/2} s on the excited surface, then
// <chi_e|R|chi_e> and <chi_e|chi_e> per molecule (FP64 reduction)
// ----------------------------------------------------------------------------
namespace ms {

template <int NR>
__global__ void __launch_bounds__(FFTShape<NR>::THREADS)
    mol_observe_kernel(SpeciesDev sp, MolDev md, int RB) {
  constexpr int NRP = NR + kPad;
  extern __shared__ float4 smem4[];
  float2* s_tw = reinterpret_cast<float2*>(smem4);
  float2* s_kh = s_tw + NR;
  float2* st = s_kh + NR;
  __shared__ double s_red[8][2];
  const int lm = blockIdx.x;
  const int m = sp.mol[lm];
  for (int q = threadIdx.x; q < NR; q += blockDim.x) {
    s_tw[q] = __ldg(&sp.twiddle[q]);
    s_kh[q] = __ldg(&sp.khalf[q]);
  }
  const int ne = sp.rows - sp.rows_g;  // excited rows
  const float2* ge = sp.psi + ((long long)lm * sp.rows + sp.rows_g) * NR;
  double num = 0.0, den = 0.0;
  for (int b0 = 0; b0 < ne; b0 += RB) {  // blocks of RB rows
    const int nb = min(RB, ne - b0);
    __syncthreads();
    load_state(st, ge + (long long)b0 * NR, nb, NR, NRP);
    __syncthreads();
    kinetic_pass<NR>(st, nb, s_kh, s_tw);  // psi = T^{1/2} s
    for (int r = threadIdx.x; r < NR; r += blockDim.x) {
      float a = 0.f;
      for (int row = 0; row < nb; ++row) {
        const float2 v = st[row * NRP + r];
        a = fmaf(v.x, v.x, fmaf(v.y, v.y, a));
      }
      den += (double)a;
      num += (double)a * (double)__ldg(&sp.r[r]);
    }
  }
  num = warp_sum(num);
  den = warp_sum(den);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) {
    s_red[wid][0] = num;
    s_red[wid][1] = den;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0.0, b = 0.0;
    for (int ww = 0; ww < (int)(blockDim.x >> 5); ++ww) {
      a += s_red[ww][0];
      b += s_red[ww][1];
    }
    md.Rnum[m] = a * sp.dR;
    md.Rden[m] = b * sp.dR;
  }
}

// initial condition: the same radial row (ground surface, j = m = 0) for
// every molecule of a species; the rest of the state is already zero
__global__ void broadcast_row_kernel(float2* psi, const float2* row, int nr, size_t per, long long nmol) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= nmol * nr) return;
  const long long m = i / nr;
  const int a = (int)(i - m * nr);
  psi[m * per + a] = row[a];
}

cudaError_t launch_broadcast_row(float2* psi, const float2* row, int nr, size_t per, long long nmol,
                                 cudaStream_t s) {
  if (nmol == 0) return cudaSuccess;
  const long long n = nmol * nr;
  broadcast_row_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(psi, row, nr, per, nmol);
  return cudaGetLastError();
}

// ----------------------------------------------------------------------------
// streaming form, first pass: d2 = (T - 1) s for blocks of rows (rows of all
// molecules of a species are independent here); one bulk copy per block
// ----------------------------------------------------------------------------
template <int NR>
__global__ void __launch_bounds__(FFTShape<NR>::THREADS)
    mol_kinetic_kernel(SpeciesDev sp, long long rows_total, int RB, int* err) {
  extern __shared__ float4 smem4[];
  float2* s_tw = reinterpret_cast<float2*>(smem4);
  float2* s_kd = s_tw + NR;
  float2* st = s_kd + NR;
  __shared__ __align__(8) unsigned long long s_bar;
  const long long r0 = blockIdx.x * (long long)RB;
  const int nrows = (int)min((long long)RB, rows_total - r0);
  const int t = threadIdx.x;
  if (t == 0) {
    mbar_init(&s_bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  if (t == 0) {
    mbar_expect_tx(&s_bar, (unsigned)(nrows * NR * sizeof(float2)));
    bulk_g2s(st, sp.psi + r0 * NR, (unsigned)(nrows * NR * sizeof(float2)), &s_bar);
  }
  for (int q = t; q < NR; q += blockDim.x) {
    s_tw[q] = __ldg(&sp.twiddle[q]);
    s_kd[q] = __ldg(&sp.kdelta[q]);
  }
  const bool ok = mbar_wait(&s_bar, 0, kWaitPolls);
  if (!__syncthreads_and(ok)) {
    if (t == 0) atomicOr(err, kErrTimeout);
    if (!ok) mbar_wait(&s_bar, 0, kWaitPolls);
    return;
  }
  kinetic_pass<NR>(st, nrows, s_kd, s_tw);
  const float4* s4 = reinterpret_cast<const float4*>(st);
  float4* d4 = reinterpret_cast<float4*>(sp.d2 + r0 * NR);
  for (int q = t; q < nrows * NR / 2; q += blockDim.x) d4[q] = s4[q];
}

size_t mol_state_smem(int nr, int rows) { return (size_t)rows * (nr + kPad) * sizeof(float2); }

static int threads_for(int nr) { return nr == 256 ? 256 : 128; }

static size_t step_smem(int nr, int nrot, int ch, bool fused) {
  const int rows = 2 * nrot;
  const int jm = (int)std::lround(std::sqrt((double)nrot)) - 1;
  const size_t nd = fused ? 0 : rows;
  return (fused ? 2 * (size_t)nr * sizeof(float2) + mol_state_smem(nr, rows) : 0) +
         2 * (size_t)rows * ch * sizeof(float2) +
         2 * (size_t)(rows + nd + 4 * (jm + 1) + 1) * ch * sizeof(float2) +
         2 * (size_t)nrot * kMaxCoupl * sizeof(int2) + (size_t)rows * sizeof(int2);
}

// rows each thread owns at chunk width ch (8 warps; 32/ch row groups per warp)
static int rows_per_thread(int nrot, int ch) {
  const int rstep = 8 * (32 / ch);
  return (2 * nrot + rstep - 1) / rstep;
}

// Launch shape of one species: chunk width, rows-per-thread bound, shared
// memory.  Fused: the widest chunk keeping two CTAs per SM.  Streaming: the
// widest chunk with at most 4 rows per thread (64 registers, four CTAs per
// SM), else at most 12.
struct StepShape {
  int ch, maxr;
  size_t smem;
  bool ok;
};
static StepShape step_shape(int nr, int nrot, bool fused) {
  // k CTAs per SM: k x (dynamic + static (< 800 B) + 1 KB reserved) <= 228 KB
  auto cap = [](int k) { return (size_t)(228 * 1024 / k - 1024 - 800); };
  if (fused) {
    for (int k : {2, 1})
      for (int ch = kChunk; ch >= 8; ch >>= 1)
        if (rows_per_thread(nrot, ch) <= 12 && step_smem(nr, nrot, ch, true) <= cap(k))
          return {ch, 12, step_smem(nr, nrot, ch, true), true};
    return {8, 12, 0, false};
  }
  for (int maxr : {4, 12, 24})
    for (int ch = kChunk; ch >= 4; ch >>= 1)
      if (rows_per_thread(nrot, ch) <= maxr &&
          step_smem(nr, nrot, ch, false) <= cap(maxr == 4 ? 4 : (maxr == 12 ? 2 : 1)))
        return {ch, maxr, step_smem(nr, nrot, ch, false), true};
  return {4, 24, 0, false};
}

bool mol_step_supported(int nr, int nrot, int path) {
  return step_shape(nr, nrot, path == MS_MOL_FUSED).ok;
}

// The chunked kernel's launch shape at a given chunk width (the plan a tuner
// picked), or ok = false where that width does not fit.
static StepShape step_shape_ch(int nr, int nrot, bool fused, int ch) {
  auto cap = [](int k) { return (size_t)(228 * 1024 / k - 1024 - 800); };
  if (ch != 4 && ch != 8 && ch != 16 && ch != 32) return {ch, 12, 0, false};
  if (fused) {
    const size_t sm = step_smem(nr, nrot, ch, true);
    return {ch, 12, sm, ch >= 8 && rows_per_thread(nrot, ch) <= 12 && sm <= cap(1)};
  }
  for (int maxr : {4, 12, 24})
    if (rows_per_thread(nrot, ch) <= maxr && step_smem(nr, nrot, ch, false) <= cap(maxr == 4 ? 4 : (maxr == 12 ? 2 : 1)))
      return {ch, maxr, step_smem(nr, nrot, ch, false), true};
  return {ch, 24, 0, false};
}

// The tiled R-space kernel covers J <= 8 (rows <= 162) at tile widths of 32
// and 16 radial points (N_r 64, 128 and 256 hold an even number of tiles).
// Its static rule: 16-point tiles from J = 5 on (two CTAs per SM), else 32.
static bool rspace_ok(int nr, int jmax) { return (nr == 64 || nr == 128 || nr == 256) && jmax <= 16; }
static int rspace_tile(const SpeciesDev& sp) {
  if (sp.jmax >= 9) return 8;
  if (sp.kern == MS_KERN_TILE && (sp.ch == 16 || sp.ch == 32)) return sp.ch;
  return sp.jmax >= 5 ? 16 : 32;
}

// The plans a species can run: (layout, kernel, chunk width).  Parity-reduced
// and d(R) species have one (the point-resident kernel); the mixed kinetic
// pass needs the streaming layout.
int mol_plan_candidates(const SpeciesDev& sp, int (*out)[4], int max) {
  int n = 0;
  auto add = [&](int path, int kern, int ch, int cps = 0) {
    if (n < max) {
      out[n][0] = path;
      out[n][1] = kern;
      out[n][2] = ch;
      out[n][3] = cps;
    }
    ++n;
  };
  if (sp.bloch || sp.par || sp.dipw) return 0;
  if (!sp.mixed) {
    if (sp.nr == 128 && sp.jmax <= 4) add(MS_MOL_FUSED, MS_KERN_POINT, 0);
    for (int ch : {32, 16, 8})
      if (step_shape_ch(sp.nr, sp.nrot, true, ch).ok) add(MS_MOL_FUSED, MS_KERN_CHUNK, ch);
  }
  if (sp.jmax <= 4) add(MS_MOL_STREAMING, MS_KERN_POINT, 0);
  if (rspace_ok(sp.nr, sp.jmax)) {  // tile width x grid: as many CTAs as fit, one per SM, one per molecule
    if (sp.jmax >= 9) {
      for (int cps : {0, -1}) add(MS_MOL_STREAMING, MS_KERN_TILE, 8, cps);
    } else {
      for (int tile : {32, 16})
        for (int cps : {0, 1, -1}) add(MS_MOL_STREAMING, MS_KERN_TILE, tile, cps);
    }
  }
  if (pair_ok(sp.nr, sp.jmax)) {  // two points a thread: 32 or 16 for J <= 4, 16 or 8 to J = 8, then 8
    if (sp.jmax >= 9) {
      for (int cps : {0, 1, -1}) add(MS_MOL_STREAMING, MS_KERN_PAIR, 8, cps);
    } else {
      for (int tile : {sp.jmax <= 4 ? 32 : 16, sp.jmax <= 4 ? 16 : 8})
        for (int cps : {0, 1, -1}) add(MS_MOL_STREAMING, MS_KERN_PAIR, tile, cps);
    }
  }
  for (int ch : {32, 16, 8, 4})
    if (step_shape_ch(sp.nr, sp.nrot, false, ch).ok) add(MS_MOL_STREAMING, MS_KERN_CHUNK, ch);
  return n < max ? n : max;
}

// cuTensorMapEncodeTiled, looked up once through the runtime
static PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    else
      cudaGetLastError();
  });
  return fn;
}

// [nrows][nr] array of complex FP32 values (8-byte elements), box tile x box_rows
static bool encode_rows(CUtensorMap* m, const void* base, unsigned long long nr, unsigned long long nrows,
                        unsigned box_rows, unsigned tile) {
  const PFN_cuTensorMapEncodeTiled_v12000 fn = tensor_map_encoder();
  if (!fn || !base) return false;
  const cuuint64_t dims[2] = {nr, nrows};
  const cuuint64_t strides[1] = {nr * sizeof(float2)};
  const cuuint32_t box[2] = {(cuuint32_t)tile, box_rows};
  const cuuint32_t es[2] = {1, 1};
  return fn(m, CU_TENSOR_MAP_DATA_TYPE_INT64, 2, const_cast<void*>(base), dims, strides, box, es,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// The species' tensor maps, encoded on first use of a given set of arrays
// (a few entries are kept: each handle, and the allocation-free scratch).
static bool rspace_maps(const SpeciesDev& sp, int tile, bool pair, RspaceMaps* out) {
  struct Entry {
    const void *psi, *d2, *vd, *vh, *mk;
    int nmol, nr, rows, tile;
    RspaceMaps maps;
  };
  static std::mutex mu;
  static std::vector<Entry> cache;
  std::lock_guard<std::mutex> lock(mu);
  // the pair kernel reads the potential and mask tables in its pair layout
  const float2 *vd = pair ? sp.vdelta_pp : sp.vdelta, *vh = pair ? sp.vhalf_pp : sp.vhalf,
               *mk = pair ? sp.maskw_pp : sp.maskw;
  for (const Entry& e : cache)
    if (e.psi == sp.psi && e.d2 == sp.d2 && e.vd == vd && e.vh == vh && e.mk == mk && e.nmol == sp.nmol &&
        e.nr == sp.nr && e.rows == sp.rows && e.tile == tile) {
      *out = e.maps;
      return true;
    }
  Entry e{sp.psi, sp.d2, vd, vh, mk, sp.nmol, sp.nr, sp.rows, tile, {}};
  const unsigned rows = sp.rows, nv = 2 * (sp.jmax + 1);  // stored rows a molecule (parity-reduced: half)
  const unsigned boxr = rows < 256 ? rows : 256, lastr = rows - (rows + boxr - 1) / boxr * boxr + boxr;
  const unsigned long long nr = sp.nr, nrows = (unsigned long long)sp.nmol * rows;
  if (!encode_rows(&e.maps.s, sp.psi, nr, nrows, boxr, tile) || !encode_rows(&e.maps.d2, sp.d2, nr, nrows, boxr, tile) ||
      !encode_rows(&e.maps.s_r, sp.psi, nr, nrows, lastr, tile) ||
      !encode_rows(&e.maps.d2_r, sp.d2, nr, nrows, lastr, tile) ||
      !encode_rows(&e.maps.vd, vd, nr, nv, nv, tile) || !encode_rows(&e.maps.vh, vh, nr, nv, nv, tile) ||
      !encode_rows(&e.maps.mk, mk, nr, 1, 1, tile))
    return false;
  if (cache.size() >= 32) cache.erase(cache.begin());
  cache.push_back(e);
  *out = e.maps;
  return true;
}

bool mol_tensor_maps_available() { return tensor_map_encoder() != nullptr; }

// rows per kinetic block: 32 KB of state
static int kinetic_rows(int nr) { return 4096 / nr; }

template <int NR, bool FUSED, int MAXR>
static void launch_step_tt(const SpeciesDev& sp, const MolDev& md, const Grid& g, int prescribed, int* err,
                           const StepShape& sh, cudaStream_t s) {
  auto k = mol_step_kernel<NR, FUSED, MAXR>;
  cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sh.smem);
  k<<<sp.nmol, FFTShape<NR>::THREADS, sh.smem, s>>>(sp, md, g, prescribed, sh.ch, err);
}

// ----------------------------------------------------------------------------
// Mixed form of the kinetic pass: d2 = (K - I) s for every row as a tensor-core
// GEMM on split FP16 operands (x = x_hi + x_lo, three products, FP32
// accumulation in tensor memory).  K is the N_r x N_r circulant of the
// kinetic propagator (symmetric).  Transposed so that the accumulator lanes
// are radial points: D[n][m] = sum_k (K - I)[n][k] s_m[k], A = K - I (resident
// in shared memory, four planes), B = 64 state rows per tile (four planes,
// double buffered), D double-buffered in tensor memory: one tile is staged
// while the previous tile's products run, and written out while the next
// tile's run.  K - I being circulant, its K-slice j (columns 16 j..16 j + 15)
// is slice 0 with the rows shifted by 16 j; A is therefore stored once as
// one 16-column strip of 128 + N_r - 16 rows, and slice j is the window
// starting 16 j rows higher.
// ----------------------------------------------------------------------------
__host__ __device__ inline int tc_kmaj_off(int r, int k, int K) {
  // K-major, no swizzle: 8-row x 16-byte core matrices, 128 B each, row groups outer
  return ((r >> 3) * (K >> 3) + (k >> 3)) * 128 + (r & 7) * 16 + (k & 7) * 2;
}
int mixed_plane_offset(int row, int k, int nr) { return tc_kmaj_off(row, k, 16); }
int mixed_strip_rows(int nr) { return 128 + nr - 16; }
bool mol_mixed_supported(int nr) { return nr == 64 || nr == 128; }

// shared-memory matrix descriptor: start, leading (K-direction) and stride
// (8-row group) byte offsets, no swizzle
__device__ __forceinline__ unsigned long long tc_desc(unsigned addr, unsigned lbo, unsigned sbo) {
  return (unsigned long long)((addr >> 4) & 0x3FFF) | ((unsigned long long)((lbo >> 4) & 0x3FFF) << 16) |
         ((unsigned long long)((sbo >> 4) & 0x3FFF) << 32) | (1ull << 46);
}
__device__ __forceinline__ void tc_mma(unsigned d, unsigned long long a, unsigned long long b, unsigned idesc,
                                       int accumulate) {
  asm volatile(
      "{ .reg .pred p; setp.ne.b32 p, %4, 0; tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p; }" ::"r"(d),
      "l"(a), "l"(b), "r"(idesc), "r"(accumulate));
}
__device__ __forceinline__ void tc_ld32(unsigned taddr, unsigned (&v)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
        "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]),
        "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]),
        "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
      : "r"(taddr));
}

template <int NR>
struct TcShape {
  static constexpr int MR = 128;                 // accumulator lanes: radial points (>= NR discarded)
  static constexpr int TR = 64;                  // state rows per tile (the MMA's N)
  static constexpr int KS = NR / 16;             // K slices of 16
  static constexpr int SR = MR + NR - 16;        // rows of the circulant strip
  static constexpr int APL = SR * 16 * 2;        // bytes of one strip plane
  static constexpr int BPL = TR * NR * 2;        // bytes of one B plane
  static constexpr int LOADS = TR * NR / (256 * 2);  // 16-byte loads per thread per tile
  static constexpr int SMEM = 4 * APL + 2 * 4 * BPL; // strip + two tile buffers
};

template <int NR>
__global__ void __launch_bounds__(256, 1) mol_kinetic_tc_kernel(SpeciesDev sp, long long rows, int* err) {
  using S = TcShape<NR>;
  constexpr int TR = S::TR, KS = S::KS, APL = S::APL, BPL = S::BPL, LOADS = S::LOADS;
  constexpr unsigned SBO_A = 2 * 128, SBO_B = (NR / 8) * 128;
  constexpr unsigned kCols = 4 * TR;  // tensor memory: 2 buffers x (Re, Im) x TR rows
  extern __shared__ __align__(1024) uint8_t smem_tc[];
  uint8_t* A = smem_tc;             // (K - I) strip: Re hi, Re lo, Im hi, Im lo
  uint8_t* Bt = smem_tc + 4 * APL;  // two tile buffers, each Re hi, Re lo, Im hi, Im lo
  __shared__ __align__(8) unsigned long long bar[2];  // [0] A staged, [1] products done
  __shared__ unsigned tmem_base;
  __shared__ float s_wmax[8][TR];                       // per warp: row maxima of the tile being staged
  __shared__ int s_rexp[2][TR];                         // per tile buffer: row scale exponents
  const int t = threadIdx.x, w = t >> 5, lane = t & 31;
  const float2* X = sp.psi;
  float2* Y = sp.d2;

  if (t == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    mbar_expect_tx(&bar[0], 4u * APL);
    bulk_g2s(A, sp.kpl, 4u * APL, &bar[0]);
  }
  if (w == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                 "r"(kCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const unsigned tmem = tmem_base;
  auto release = [&]() {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (w == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kCols));
  };
  // a wait on bar[id] phase ph by every thread, uniform outcome; on a timeout
  // the products in flight get a second bounded wait before tensor memory is freed
  auto wait_all = [&](int id, unsigned ph) -> bool {
    const bool ok = mbar_wait_sleep(&bar[id], ph);
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (__syncthreads_and(ok)) return true;
    if (t == 0) atomicOr(err, kErrTimeout);
    if (!ok) mbar_wait_sleep(&bar[id], ph);
    release();
    return false;
  };
  if (!wait_all(0, 0)) return;

  // load slot u of a tile: rows 8 q + (lane & 7), points 8 kc + 2 (lane >> 3) (+1)
  auto slot_row = [&](int u) { return 8 * ((w + 8 * u) / (NR / 8)) + (lane & 7); };
  auto slot_k = [&](int u) { return 8 * ((w + 8 * u) % (NR / 8)) + 2 * (lane >> 3); };
  float4 pre[LOADS];
  auto fetch = [&](long long tile) {
#pragma unroll
    for (int u = 0; u < LOADS; ++u) {
      const long long gr = tile * TR + slot_row(u);
      pre[u] = gr < rows ? __ldcs(reinterpret_cast<const float4*>(X + gr * NR + slot_k(u)))
                         : make_float4(0.f, 0.f, 0.f, 0.f);
    }
  };
  // The fetched tile -> four FP16 planes of buffer buf.  Each state row is
  // scaled by 2^e so that its largest |Re|, |Im| lies in [2^14, 2^15) (an
  // exact power-of-two scale, undone on write-out): hi = fp16(x), lo =
  // fp16(x - hi) then carry 22 bits of every element of the row's scale.
  // Row maxima: slot u of every thread lies in row group u / UPQ (rows 8 q +
  // (lane & 7)) whatever the warp, so each thread folds its slots per group,
  // the four lanes sharing a row fold by shuffles, and each warp leaves one
  // value per row; 64 threads then fold the 8 warps' values.
  auto stage = [&](int buf) {
    constexpr int UPQ = LOADS / 8;
    static_assert(LOADS % 8 == 0 && TR == 64, "eight row groups of eight rows per tile");
    uint8_t* B0 = Bt + buf * 4 * BPL;
    float rm[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) rm[q] = 0.f;
#pragma unroll
    for (int u = 0; u < LOADS; ++u)
      rm[u / UPQ] = fmaxf(rm[u / UPQ], fmaxf(fmaxf(fabsf(pre[u].x), fabsf(pre[u].y)),
                                             fmaxf(fabsf(pre[u].z), fabsf(pre[u].w))));
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      rm[q] = fmaxf(rm[q], __shfl_xor_sync(0xffffffffu, rm[q], 8));
      rm[q] = fmaxf(rm[q], __shfl_xor_sync(0xffffffffu, rm[q], 16));
    }
    if (lane < 8) {
#pragma unroll
      for (int q = 0; q < 8; ++q) s_wmax[w][8 * q + lane] = rm[q];
    }
    __syncthreads();
    if (t < TR) {
      float m = 0.f;
#pragma unroll
      for (int ww = 0; ww < 8; ++ww) m = fmaxf(m, s_wmax[ww][t]);
      int ex = 0;
      if (m > 0.f) frexpf(m, &ex);
      s_rexp[buf][t] = m > 0.f ? min(15 - ex, 100) : 0;
    }
    __syncthreads();
#pragma unroll
    for (int u = 0; u < LOADS; ++u) {
      const float sc = __int_as_float((127 + s_rexp[buf][slot_row(u)]) << 23);  // 2^e
      const float re[2] = {pre[u].x * sc, pre[u].z * sc}, im[2] = {pre[u].y * sc, pre[u].w * sc};
      __half rh[2], rl[2], ih[2], il[2];
#pragma unroll
      for (int e = 0; e < 2; ++e) {
        rh[e] = __float2half_rn(re[e]);
        rl[e] = __float2half_rn(re[e] - __half2float(rh[e]));
        ih[e] = __float2half_rn(im[e]);
        il[e] = __float2half_rn(im[e] - __half2float(ih[e]));
      }
      const int off = tc_kmaj_off(slot_row(u), slot_k(u), NR);
      *reinterpret_cast<__half2*>(B0 + 0 * BPL + off) = __halves2half2(rh[0], rh[1]);
      *reinterpret_cast<__half2*>(B0 + 1 * BPL + off) = __halves2half2(rl[0], rl[1]);
      *reinterpret_cast<__half2*>(B0 + 2 * BPL + off) = __halves2half2(ih[0], ih[1]);
      *reinterpret_cast<__half2*>(B0 + 3 * BPL + off) = __halves2half2(il[0], il[1]);
    }
  };
  auto issue = [&](int buf) {  // 2 outputs x 6 split products x KS slices, one thread
    // FP32 accumulator (bit 4), A and B FP16 (format fields at bits 7 and 10 zero), N, M
    constexpr unsigned idp = (1u << 4) | ((unsigned)(TR >> 3) << 17) | ((unsigned)(128 >> 4) << 24);
    constexpr unsigned idn = idp | (1u << 14);  // B negated
    // {A plane, B plane, negate}: Re = Kr Xr - Ki Xi, Im = Kr Xi + Ki Xr, each as hh + hl + lh
    constexpr int blk[2][6][3] = {{{0, 0, 0}, {0, 1, 0}, {1, 0, 0}, {2, 2, 1}, {2, 3, 1}, {3, 2, 1}},
                                  {{0, 2, 0}, {0, 3, 0}, {1, 2, 0}, {2, 0, 0}, {2, 1, 0}, {3, 0, 0}}};
    // slice j: A window starts (NR - 16 - 16 j) rows into the strip, B at column 16 j
    unsigned long long da[4], db[4];
#pragma unroll
    for (int p = 0; p < 4; ++p) {
      da[p] = tc_desc(smem_u32(A + p * APL) + ((NR - 16) / 8) * SBO_A, 128, SBO_A);
      db[p] = tc_desc(smem_u32(Bt + (buf * 4 + p) * BPL), 128, SBO_B);
    }
#pragma unroll
    for (int o = 0; o < 2; ++o) {
      const unsigned d = tmem + (unsigned)(buf * 2 * TR + o * TR);
#pragma unroll
      for (int b = 0; b < 6; ++b)
#pragma unroll
        for (int j = 0; j < KS; ++j)
          tc_mma(d, da[blk[o][b][0]] - (unsigned long long)(j * 2 * SBO_A / 16),
                 db[blk[o][b][1]] + (unsigned long long)(j * 256 / 16), blk[o][b][2] ? idn : idp,
                 (b | j) != 0);
    }
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                     smem_u32(&bar[1]))
                 : "memory");
  };
  auto drain = [&](int buf, long long tile) {  // tensor memory -> d2 rows of the tile
    constexpr int H = TR / 2;                       // rows per warp half
    const int n = 32 * (w & 3) + lane, rh = w >> 2;  // radial point, row half
    static_assert(H == 32, "the write-out loads 32 accumulator columns per warp half");
    unsigned re[H], im[H];
    const unsigned ta = tmem + ((unsigned)(32 * (w & 3)) << 16) + (unsigned)(buf * 2 * TR + H * rh);
    tc_ld32(ta, re);
    tc_ld32(ta + TR, im);
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
    if (n < NR) {
#pragma unroll
      for (int r = 0; r < H; ++r) {
        const long long gr = tile * TR + H * rh + r;
        // undo the row's and the matrix's power-of-two scales
        const float us = __int_as_float((127 - s_rexp[buf][H * rh + r] - sp.kpl_exp) << 23);
        if (gr < rows)
          __stcs(Y + gr * NR + n, make_float2(__uint_as_float(re[r]) * us, __uint_as_float(im[r]) * us));
      }
    }
  };
  auto sync_async = [&]() {  // the staged planes are visible to the tensor cores
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  };

  // tile i: staged into buffer i & 1 while the products of tile i - 1 run
  // (its loads were issued one iteration earlier), issued once those are
  // done; then tile i - 1 is written out while tile i's products run
  const long long ntiles = (rows + TR - 1) / TR;
  long long tile = blockIdx.x;
  if (tile >= ntiles) {
    release();
    return;
  }
  fetch(tile);
  stage(0);
  sync_async();
  if (t == 0) issue(0);
  long long prev = tile;
  tile += gridDim.x;
  if (tile < ntiles) fetch(tile);
  int i = 1;
  for (; tile < ntiles; tile += gridDim.x, ++i) {
    stage(i & 1);  // buffer i & 1 was read by the products of tile i - 2, complete
    if (tile + gridDim.x < ntiles) fetch(tile + gridDim.x);  // in flight until the next stage
    sync_async();
    if (!wait_all(1, (unsigned)((i - 1) & 1))) return;  // products of tile i - 1
    if (t == 0) issue(i & 1);
    drain((i - 1) & 1, prev);  // overlaps the products of tile i
    prev = tile;
  }
  if (!wait_all(1, (unsigned)((i - 1) & 1))) return;
  drain((i - 1) & 1, prev);
  release();
}

// Stage 1 of a species' step: in the streaming form the per-molecule field
// records (point-resident R-space kernel only) and the kinetic pass d2 = (T - 1) s.
// Stage 2: the R-space pass (streaming form) or the whole fused step.
// Each returns the number of kernels it launched.
template <int NR>
static int launch_stage1_t(const SpeciesDev& sp, const MolDev& md, const Grid& g, int prescribed, int* err,
                           cudaStream_t s) {
  if (sp.path == MS_MOL_FUSED) {
    if (!use_point(sp)) return 0;
    mol_field_kernel<<<(sp.nmol + 127) / 128, 128, 0, s>>>(sp, md, g, prescribed, err);
    return 1;
  }
  int n = 0;
  if (use_point(sp) || use_tile(sp) || use_pair(sp)) {  // the per-molecule frame-field records those kernels read
    mol_field_kernel<<<(sp.nmol + 127) / 128, 128, 0, s>>>(sp, md, g, prescribed, err);
    ++n;
  }
  const long long rows_total = (long long)sp.nmol * sp.rows;
  if (sp.mixed) {  // split-FP16 tensor-core GEMM
    if constexpr (NR == 64 || NR == 128) {
      using T = TcShape<NR>;
      int dev = 0, nsm = 0;
      cudaGetDevice(&dev);
      cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
      const long long ntiles = (rows_total + T::TR - 1) / T::TR;
      const int grid = (int)std::min<long long>(ntiles, (long long)(nsm > 0 ? nsm : 1));
      cudaFuncSetAttribute(mol_kinetic_tc_kernel<NR>, cudaFuncAttributeMaxDynamicSharedMemorySize, T::SMEM);
      mol_kinetic_tc_kernel<NR><<<grid, 256, T::SMEM, s>>>(sp, rows_total, err);
    }
    return n + 1;
  }
  const int RB = kinetic_rows(NR);
  const size_t ksmem = 2 * (size_t)NR * sizeof(float2) + (size_t)RB * NR * sizeof(float2);
  cudaFuncSetAttribute(mol_kinetic_kernel<NR>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ksmem);
  mol_kinetic_kernel<NR><<<(unsigned)((rows_total + RB - 1) / RB), FFTShape<NR>::THREADS, ksmem, s>>>(
      sp, rows_total, RB, err);
  return n + 1;
}

template <int NR>
static int launch_stage2_t(const SpeciesDev& sp, const MolDev& md, const Grid& g, int prescribed, int* err,
                           cudaStream_t s) {
  const bool fused = sp.path == MS_MOL_FUSED;
  const StepShape sh = sp.kern == MS_KERN_CHUNK && sp.ch > 0 ? step_shape_ch(NR, sp.nrot, fused, sp.ch)
                                                             : step_shape(NR, sp.nrot, fused);
  if (fused) {
    if constexpr (NR == 128) {
      if (use_point(sp)) {
        launch_rpoint_n<NR, true>(sp, md, err, s);
        if (sp.dipw) launch_dipole_r<NR>(sp, md, err, s);
        return sp.dipw ? 2 : 1;
      }
    }
    launch_step_tt<NR, true, 12>(sp, md, g, prescribed, err, sh, s);
    return 1;
  }
  if (use_point(sp)) {  // point-resident R-space pass
    launch_rpoint_n<NR>(sp, md, err, s);
    if constexpr (NR <= 128) {
      if (sp.dipw) {
        launch_dipole_r<NR>(sp, md, err, s);
        return 2;
      }
    }
    return 1;
  }
  RspaceMaps maps;
  if (use_pair(sp)) {
    if (rspace_maps(sp, pair_tile(sp), true, &maps)) {
      launch_rspace_pair(sp, md, err, maps, pair_tile(sp), s);
      return 1;
    }
    if (sp.par) {  // no other kernel takes the parity-reduced state beyond J = 4: report it
      flag_error_kernel<<<1, 1, 0, s>>>(err, kErrLaunch);
      return 1;
    }
  }
  if (use_tile(sp) && rspace_maps(sp, rspace_tile(sp), false, &maps)) {
    launch_rspace(sp, md, err, maps, rspace_tile(sp), s);
    return 1;
  }
  if (sh.maxr == 4) launch_step_tt<NR, false, 4>(sp, md, g, prescribed, err, sh, s);
  else if (sh.maxr == 12) launch_step_tt<NR, false, 12>(sp, md, g, prescribed, err, sh, s);
  else launch_step_tt<NR, false, 24>(sp, md, g, prescribed, err, sh, s);
  return 1;
}

int launch_mol_stage1(const SpeciesDev& sp, const MolDev& md, const Grid& g, int prescribed, int* err,
                      cudaStream_t s) {
  if (sp.nmol == 0 || sp.bloch) return 0;
  switch (sp.nr) {
    case 64: return launch_stage1_t<64>(sp, md, g, prescribed, err, s);
    case 128: return launch_stage1_t<128>(sp, md, g, prescribed, err, s);
    case 256: return launch_stage1_t<256>(sp, md, g, prescribed, err, s);
  }
  return 0;
}

int launch_mol_stage2(const SpeciesDev& sp, const MolDev& md, const Grid& g, int prescribed, int* err,
                      cudaStream_t s) {
  if (sp.nmol == 0) return 0;
  if (sp.bloch) return launch_bloch_step(sp, md, g, prescribed, err, s);
  switch (sp.nr) {
    case 64: return launch_stage2_t<64>(sp, md, g, prescribed, err, s);
    case 128: return launch_stage2_t<128>(sp, md, g, prescribed, err, s);
    case 256: return launch_stage2_t<256>(sp, md, g, prescribed, err, s);
  }
  return 0;
}

template <int NR>
static void launch_observe_t(const SpeciesDev& sp, const MolDev& md, cudaStream_t s) {
  const int RB = min(sp.nrot, 4096 / NR);
  const size_t smem = 2 * (size_t)NR * sizeof(float2) + mol_state_smem(NR, RB);
  cudaFuncSetAttribute(mol_observe_kernel<NR>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  mol_observe_kernel<NR><<<sp.nmol, FFTShape<NR>::THREADS, smem, s>>>(sp, md, RB);
}

void launch_mol_observe(const SpeciesDev& sp, const MolDev& md, cudaStream_t s) {
  if (sp.nmol == 0) return;
  if (sp.bloch) {
    launch_bloch_observe(sp, md, s);
    return;
  }
  switch (sp.nr) {
    case 64: launch_observe_t<64>(sp, md, s); break;
    case 128: launch_observe_t<128>(sp, md, s); break;
    case 256: launch_observe_t<256>(sp, md, s); break;
  }
}

}  // namespace ms
