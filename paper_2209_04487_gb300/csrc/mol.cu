// Molecular split-operator step (Eqs. 3-5 with the surfaces of Eqs. 6-7),
// one CTA per molecule, the molecule's whole state resident in shared memory.
//
// The library stores phi = T^{1/2} psi, so that one coupled step is
//   chi  = Mask V^{1/2} K(E') V^{1/2} phi      (R-space pass, per radial point)
//   phi' = T chi                               (kinetic pass, per channel)
// which equals the paper's split-operator step T^{1/2} Mask V^{1/2} K V^{1/2}
// T^{1/2} on psi (T commutes with the angular coupling because the
// transition dipole is R-independent, and is unitary per channel, so
// populations and the dipole can be taken from chi).
//
// Norm-preserving FP32 arithmetic: every unit-modulus factor (potential
// phase, kinetic phase, FFT twiddle) is carried as an FP32 hi+lo pair and
// applied with a compensated product, so the factor is exact to ~1e-15 and
// only unbiased output rounding remains.  Every factor of the step is close
// to the identity (|V dtau| and |k^2 dtau/2mu| are a few 1e-2), so the step
// is computed as a correction: d1 = (V - 1) phi + V^{1/2} S with
// S = sum_{n>=1} (i theta sigma_x M)^n/n! V^{1/2} phi (Taylor series of the
// coupling exponential, |theta M| << 1), chi = phi + d1,
// d2 = (T - 1) chi, and phi' = phi + (d1 + d2): the full-magnitude state is
// rounded once per step, which keeps the FP32 norm error a random walk of
// about 1e-8 per step instead of a drift.
#include "ms_internal.cuh"

namespace ms {

namespace {

constexpr int kPad = 8;  // row padding (float2): keeps rows 16-byte aligned and banks spread

template <int NR>
struct FFTShape;
template <>
struct FFTShape<64> {
  static constexpr int N1 = 8, N2 = 8, THREADS = 128;
};
template <>
struct FFTShape<128> {
  static constexpr int N1 = 16, N2 = 8, THREADS = 128;
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
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ float2 operator+(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 operator-(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }

// multiply by exp(-+ i t pi/8) (forward: minus)
template <int T, bool INV>
__device__ __forceinline__ float2 twiddle16(float2 v) {
  if constexpr (T == 0) {
    return v;
  } else if constexpr (T == 4) {
    return INV ? make_float2(-v.y, v.x) : make_float2(v.y, -v.x);
  } else {
    constexpr double c = cos_pi8(T);
    constexpr double s = INV ? sin_pi8(T) : -sin_pi8(T);
    return cmul_c(v, hi_of(c), hi_of(s), lo_of(c), lo_of(s));
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

// Four-step FFT kinetic pass on all `rows` rows (each NR complex, stride
// NRP) held in shared memory: forward DFT, multiply by kph[k], inverse DFT.
// n = n1 + N1 n2, k = k2 + N2 k1.  Step A: per n1, an N2-point DFT over n2
// and the twiddle exp(-2 pi i n1 k2/NR); step B: per k2, an N1-point DFT
// over n1.  Intermediate y[n1][k2] lives at n1 + N1 k2 (xor-swizzled within
// each block of N1 so that step B is bank-conflict free).
// MODE kInPlace: st <- T st (kph = full phases / NR).
// MODE kDeltaOut: st holds chi = phi + d1 and D holds d1; with kph the
// phase deltas (P_k - 1)/NR the pass forms d2 = (T - 1) chi and writes
// phi' = phi + (d1 + d2) to gout, where gout still holds phi: the whole
// step reaches the stored state through a single FP32 rounding.
enum { kInPlace = 0, kDeltaOut = 1 };

template <int NR, int MODE>
__device__ void kinetic_pass(float2* st, int rows, const float4* __restrict__ kph,
                             const float4* __restrict__ tw, float2* gout, const float2* D) {
  using S = FFTShape<NR>;
  constexpr int N1 = S::N1, N2 = S::N2, NT = S::THREADS, NRP = NR + kPad;
  const int t = threadIdx.x;
  // ---- step A: rows processed NT/N1 at a time
  {
    constexpr int per = NT / N1;
    const int n1 = t % N1, rsub = t / N1;
    for (int r0 = 0; r0 < rows; r0 += per) {
      const int row = r0 + rsub;
      float2 x[N2];
      if (row < rows) {
#pragma unroll
        for (int n2 = 0; n2 < N2; ++n2) x[n2] = st[row * NRP + n1 + N1 * n2];
      }
      __syncthreads();
      if (row < rows) {
        dft_reg<N2, false>(x);
#pragma unroll
        for (int k2 = 0; k2 < N2; ++k2) {
          const float4 w = __ldg(&tw[n1 * N2 + k2]);
          const float2 y = cmul_c(x[k2], w.x, w.y, w.z, w.w);
          st[row * NRP + (n1 ^ (k2 % N1)) + N1 * k2] = y;
        }
      }
      __syncthreads();
    }
  }
  // ---- step B (+ kinetic phase + inverse step B), in place per thread
  {
    constexpr int per = NT / N2;
    const int k2 = t % N2, rsub = t / N2;
    for (int r0 = 0; r0 < rows; r0 += per) {
      const int row = r0 + rsub;
      if (row < rows) {
        float2 x[N1];
#pragma unroll
        for (int n1 = 0; n1 < N1; ++n1) x[n1] = st[row * NRP + (n1 ^ (k2 % N1)) + N1 * k2];
        dft_reg<N1, false>(x);  // x[k1] = X[k2 + N2 k1]
#pragma unroll
        for (int k1 = 0; k1 < N1; ++k1) {
          const float4 p = __ldg(&kph[k2 + N2 * k1]);
          x[k1] = cmul_c(x[k1], p.x, p.y, p.z, p.w);
        }
        dft_reg<N1, true>(x);   // x[n1] = y'[n1][k2]
#pragma unroll
        for (int n1 = 0; n1 < N1; ++n1) st[row * NRP + (n1 ^ (k2 % N1)) + N1 * k2] = x[n1];
      }
    }
  }
  __syncthreads();
  // ---- inverse step A
  {
    constexpr int per = NT / N1;
    const int n1 = t % N1, rsub = t / N1;
    for (int r0 = 0; r0 < rows; r0 += per) {
      const int row = r0 + rsub;
      float2 x[N2];
      if (row < rows) {
#pragma unroll
        for (int k2 = 0; k2 < N2; ++k2) {
          const float4 w = __ldg(&tw[n1 * N2 + k2]);
          x[k2] = cmul_c(st[row * NRP + (n1 ^ (k2 % N1)) + N1 * k2], w.x, -w.y, w.z, -w.w);
        }
        dft_reg<N2, true>(x);  // x[n2] = x'[n1 + N1 n2]
      }
      if constexpr (MODE == kDeltaOut) {
        if (row < rows) {
#pragma unroll
          for (int n2 = 0; n2 < N2; ++n2) {
            const int p = n1 + N1 * n2;
            const float2 d1 = D[row * NRP + p];
            const float2 ph = gout[(long long)row * NR + p];
            const float2 dd = make_float2(d1.x + x[n2].x, d1.y + x[n2].y);
            gout[(long long)row * NR + p] = make_float2(ph.x + dd.x, ph.y + dd.y);
          }
        }
      } else {
        __syncthreads();
        if (row < rows) {
#pragma unroll
          for (int n2 = 0; n2 < N2; ++n2) st[row * NRP + n1 + N1 * n2] = x[n2];
        }
        __syncthreads();
      }
    }
  }
}

__device__ __forceinline__ void load_state(float2* st, const float2* __restrict__ g, int rows, int NR,
                                           int NRP) {
  const float4* g4 = reinterpret_cast<const float4*>(g);
  const int per_row = NR / 2;
  const int total = rows * per_row;
  for (int q = threadIdx.x; q < total; q += blockDim.x) {
    const int row = q / per_row, col = q - row * per_row;
    reinterpret_cast<float4*>(st + row * NRP)[col] = g4[q];
  }
}

struct Field3 {
  float ez;      // E'_z
  float2 ep;     // E+ = (E'_x - i E'_y)/2
  float2 em;     // E- = conj(E+)
};

__device__ __forceinline__ float2 emult(const Field3& f, int kind) {
  return kind == 0 ? make_float2(f.ez, 0.f) : (kind == 1 ? f.ep : f.em);
}

// one Taylor term: out[row] = (i theta / n) * (M in_{other surface})[c]
__device__ __forceinline__ void taylor_term(const float2* __restrict__ in, float2* __restrict__ out,
                                            int nrot, int G, int t, const int4* __restrict__ cp,
                                            const Field3& f, float coef_n) {
  for (int s = 0; s < 2; ++s) {
    const int other = (1 - s) * nrot;
    for (int c = 0; c < nrot; ++c) {
      float2 acc = make_float2(0.f, 0.f);
#pragma unroll
      for (int e = 0; e < kMaxCoupl; ++e) {
        const int4 q = __ldg(&cp[c * kMaxCoupl + e]);
        if (q.x >= 0) {
          const float2 v = in[(other + q.x) * G + t];
          const float2 m = emult(f, q.y);
          const float cf = __int_as_float(q.z);
          const float2 mv = cmul(m, v);
          acc.x = fmaf(cf, mv.x, acc.x);
          acc.y = fmaf(cf, mv.y, acc.y);
        }
      }
      // multiply by i * coef_n
      out[(s * nrot + c) * G + t] = make_float2(-coef_n * acc.y, coef_n * acc.x);
    }
  }
}

}  // namespace

// ----------------------------------------------------------------------------
// the coupled molecular step
// ----------------------------------------------------------------------------
template <int NR>
__global__ void __launch_bounds__(FFTShape<NR>::THREADS)
    mol_step_kernel(SpeciesDev sp, MolDev md, Grid g, int prescribed, int G, int* err) {
  constexpr int NRP = NR + kPad;
  extern __shared__ float4 smem4[];
  float2* st = reinterpret_cast<float2*>(smem4);
  const int nrot = sp.nrot, rows = 2 * nrot;
  float2* D = st + rows * NRP;             // d1 = chi - phi (running Taylor sum first)
  float2* bufY = D + rows * NRP;           // Taylor terms, ping-pong, [rows][G]
  float2* bufZ = bufY + rows * G;
  __shared__ Field3 s_field;
  __shared__ int s_nterms;
  __shared__ double s_red[8][8];

  const int lm = blockIdx.x;
  const int m = sp.mol[lm];
  const int t = threadIdx.x;
  float2* gpsi = sp.psi + (long long)lm * rows * NR;

  load_state(st, gpsi, rows, NR, NRP);

  // ---- local field at the molecule, rotated into its frame (a.u.)
  if (t == 0) {
    float E[3];
    const long long n = *g.step;
    if (prescribed) {
      const long long nn = n < md.nwave ? n : md.nwave - 1;
      if (n >= md.nwave) atomicOr(err, kErrPrescribedRange);
      const float w = md.wave[nn];
      E[0] = md.amp[3 * (long long)m] * w;
      E[1] = md.amp[3 * (long long)m + 1] * w;
      E[2] = md.amp[3 * (long long)m + 2] * w;
    } else {
      const long long c = md.cell[m];
      E[0] = g.E[0][c];
      E[1] = g.E[1][c];
      E[2] = g.E[2][c];
    }
    const float* O = md.rot + 9 * (long long)m;  // molecule -> lab, row-major
    const float inv_fau = 1.0f / 5.14220674763e11f;
    float Ep[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) Ep[i] = (O[i] * E[0] + O[3 + i] * E[1] + O[6 + i] * E[2]) * inv_fau;
    s_field.ez = Ep[2];
    s_field.ep = make_float2(0.5f * Ep[0], -0.5f * Ep[1]);
    s_field.em = make_float2(0.5f * Ep[0], 0.5f * Ep[1]);
    // number of Taylor terms: (theta |E'|)^(n+1)/(n+1)! < 1e-13
    const double x = sp.theta * sqrt((double)Ep[0] * Ep[0] + (double)Ep[1] * Ep[1] + (double)Ep[2] * Ep[2]);
    int nt = 0;
    double term = 1.0;
    if (x > 0.0) {
      nt = 1;
      term = x;
      while (nt < 24) {
        const double next = term * x / (nt + 1);
        if (next < 1e-13) break;
        term = next;
        ++nt;
      }
      if (nt >= 24 || x > 4.0) atomicOr(err, kErrCouplingSeries);
    }
    s_nterms = nt;
  }
  __syncthreads();
  const Field3 f = s_field;
  const int nterms = s_nterms;
  const float theta = (float)sp.theta;
  const int4* __restrict__ cp = sp.coupl;

  // ---- R-space pass, G radial points at a time (thread t <-> r = r0 + t)
  double pg = 0.0, pe = 0.0, ag = 0.0, ae = 0.0, dxs = 0.0, dys = 0.0, dzs = 0.0;
  for (int r0 = 0; r0 < NR; r0 += G) {
    const int r = r0 + t;
    if (t < G) {
      // xi = V^{1/2} phi into Z; the Taylor sum S accumulates in D's column
      for (int row = 0; row < rows; ++row) {
        const int s = row / nrot, c = row - s * nrot;
        const int j = (int)sqrtf((float)c + 0.5f);  // c = j^2 + j + m
        const float2 vh = __ldg(&sp.vhalf[(s * (sp.jmax + 1) + j) * NR + r]);
        bufZ[row * G + t] = cmul(vh, st[row * NRP + r]);
        D[row * NRP + r] = make_float2(0.f, 0.f);
      }
      float2* in = bufZ;
      float2* out = bufY;
      for (int n = 1; n <= nterms; ++n) {
        taylor_term(in, out, nrot, G, t, cp, f, theta / (float)n);
        for (int row = 0; row < rows; ++row) {
          const float2 a = D[row * NRP + r], b = out[row * G + t];
          D[row * NRP + r] = make_float2(a.x + b.x, a.y + b.y);
        }
        float2* tmp = in;
        in = out;
        out = tmp;
      }
      // d1 = (V - 1) phi + V^{1/2} S ; chi = phi + d1 ; mask ; observables
      const float mk = __ldg(&sp.maskw[r]).x;
      float sg = 0.f, se = 0.f;
      double wg = 0.0, we = 0.0;
      for (int row = 0; row < rows; ++row) {
        const int s = row / nrot, c = row - s * nrot;
        const int j = (int)sqrtf((float)c + 0.5f);
        const int ti = (s * (sp.jmax + 1) + j) * NR + r;
        const float2 vh = __ldg(&sp.vhalf[ti]);
        const float4 vd = __ldg(&sp.vdelta[ti]);
        const float2 phi = st[row * NRP + r];
        float2 d1 = cmul_c_add(phi, vd, cmul(vh, D[row * NRP + r]));
        if (mk < 1.f) {
          // mask the new value: d1 <- m (phi + d1) - phi; tally the norm removed
          const double px = (double)phi.x + d1.x, py = (double)phi.y + d1.y;
          d1.x = fmaf(mk - 1.f, phi.x, mk * d1.x);
          d1.y = fmaf(mk - 1.f, phi.y, mk * d1.y);
          const double qx = (double)phi.x + d1.x, qy = (double)phi.y + d1.y;
          const double d2 = (px * px + py * py) - (qx * qx + qy * qy);
          if (s == 0) wg += d2; else we += d2;
        }
        const float2 chi = make_float2(phi.x + d1.x, phi.y + d1.y);
        const float b2 = chi.x * chi.x + chi.y * chi.y;
        if (s == 0) sg += b2; else se += b2;
        st[row * NRP + r] = chi;
        D[row * NRP + r] = d1;
      }
      // dipole in the molecule frame: sum_c conj(chi_g[c]) (A chi_e)[c]
      float2 accP = make_float2(0.f, 0.f), accM = accP, accZ = accP;
      for (int c = 0; c < nrot; ++c) {
        const float2 gc = st[c * NRP + r];
#pragma unroll
        for (int e = 0; e < kMaxCoupl; ++e) {
          const int4 q = __ldg(&cp[c * kMaxCoupl + e]);
          if (q.x >= 0) {
            const float2 ev = st[(nrot + q.x) * NRP + r];
            const float cf = __int_as_float(q.z);
            // conj(gc) * ev
            const float re = fmaf(gc.x, ev.x, gc.y * ev.y), im = fmaf(gc.x, ev.y, -gc.y * ev.x);
            float2* acc = q.y == 0 ? &accZ : (q.y == 1 ? &accP : &accM);
            acc->x = fmaf(cf, re, acc->x);
            acc->y = fmaf(cf, im, acc->y);
          }
        }
      }
      pg += sg;
      pe += se;
      ag += wg;
      ae += we;
      dxs += (double)(accP.x + accM.x);
      dys += (double)(accP.y - accM.y);
      dzs += 2.0 * (double)accZ.x;
    }
  }
  // ---- block reduction (FP64)
  {
    double v[7] = {pg, pe, ag, ae, dxs, dys, dzs};
    const int lane = t & 31, wid = t >> 5;
#pragma unroll
    for (int q = 0; q < 7; ++q) v[q] = warp_sum(v[q]);
    if (lane == 0) {
#pragma unroll
      for (int q = 0; q < 7; ++q) s_red[wid][q] = v[q];
    }
    __syncthreads();
    if (t == 0) {
      double a[7] = {0, 0, 0, 0, 0, 0, 0};
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w)
        for (int q = 0; q < 7; ++q) a[q] += s_red[w][q];
      const double dR = sp.dR;
      const double P0 = a[0] * dR, P1 = a[1] * dR;
      md.pop[2 * (long long)m] = P0;
      md.pop[2 * (long long)m + 1] = P1;
      md.absorbed[2 * (long long)m] += a[2] * dR;
      md.absorbed[2 * (long long)m + 1] += a[3] * dR;
      if (!isfinite(P0) || !isfinite(P1)) atomicOr(err, kErrNonFinite);
      // mu' = d dR (Re(S+ + S-), Im(S+ - S-), 2 Re Z), lab mu = O mu'
      const double scale = sp.dipole * dR;
      const double mup[3] = {a[4] * scale, a[5] * scale, a[6] * scale};
      const float* O = md.rot + 9 * (long long)m;
      double* mu = md.mu + 3 * (long long)m;
      double* dmu = md.dmu + 3 * (long long)m;
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        const double lab = (double)O[3 * i] * mup[0] + (double)O[3 * i + 1] * mup[1] +
                           (double)O[3 * i + 2] * mup[2];
        dmu[i] = lab - mu[i];
        mu[i] = lab;
      }
    }
  }
  __syncthreads();
  // ---- kinetic pass: phi' = phi + d1 + (T - 1) chi, written to global memory
  kinetic_pass<NR, kDeltaOut>(st, rows, sp.kdelta, sp.twiddle, gpsi, D);
}

}  // namespace ms

// ----------------------------------------------------------------------------
// Eq. 8 readout: psi = T^{-1/2} phi on the excited surface, then
// <chi_e|R|chi_e> and <chi_e|chi_e> per molecule (FP64 reduction)
// ----------------------------------------------------------------------------
namespace ms {

template <int NR>
__global__ void __launch_bounds__(FFTShape<NR>::THREADS)
    mol_observe_kernel(SpeciesDev sp, MolDev md) {
  constexpr int NRP = NR + kPad;
  extern __shared__ float4 smem4[];
  float2* st = reinterpret_cast<float2*>(smem4);
  __shared__ double s_red[8][2];
  const int nrot = sp.nrot;
  const int lm = blockIdx.x;
  const int m = sp.mol[lm];
  const float2* ge = sp.psi + ((long long)lm * 2 + 1) * nrot * NR;  // excited rows
  load_state(st, ge, nrot, NR, NRP);
  __syncthreads();
  kinetic_pass<NR, kInPlace>(st, nrot, sp.kphase_inv, sp.twiddle, nullptr, nullptr);
  double num = 0.0, den = 0.0;
  for (int r = threadIdx.x; r < NR; r += blockDim.x) {
    float a = 0.f;
    for (int row = 0; row < nrot; ++row) {
      const float2 v = st[row * NRP + r];
      a = fmaf(v.x, v.x, fmaf(v.y, v.y, a));
    }
    den += (double)a;
    num += (double)a * (double)__ldg(&sp.r[r]);
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
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
      a += s_red[w][0];
      b += s_red[w][1];
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

size_t mol_state_smem(int nr, int rows) { return (size_t)rows * (nr + kPad) * sizeof(float2); }

static int threads_for(int nr) { return nr == 256 ? 256 : 128; }

// radial points per R-space chunk so that state + d1 + 2 Taylor buffers fit
static int chunk_for(int nr, int nrot, size_t* smem) {
  const size_t cap = 227 * 1024;
  const int rows = 2 * nrot;
  const size_t base = 2 * mol_state_smem(nr, rows);
  int G = nr < threads_for(nr) ? nr : threads_for(nr);
  while (G > 8 && base + 2 * (size_t)rows * G * sizeof(float2) > cap) G >>= 1;
  *smem = base + 2 * (size_t)rows * G * sizeof(float2);
  return G;
}

size_t mol_step_smem(int nr, int nrot) {
  size_t s;
  chunk_for(nr, nrot, &s);
  return s;
}

template <int NR>
static void launch_step_t(const SpeciesDev& sp, const MolDev& md, const Grid& g, int prescribed,
                          int* err, cudaStream_t s) {
  size_t smem;
  const int G = chunk_for(NR, sp.nrot, &smem);
  cudaFuncSetAttribute(mol_step_kernel<NR>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  mol_step_kernel<NR><<<sp.nmol, FFTShape<NR>::THREADS, smem, s>>>(sp, md, g, prescribed, G, err);
}

void launch_mol_step(const SpeciesDev& sp, const MolDev& md, const Grid& g, int prescribed, int* err,
                     cudaStream_t s) {
  if (sp.nmol == 0) return;
  switch (sp.nr) {
    case 64: launch_step_t<64>(sp, md, g, prescribed, err, s); break;
    case 128: launch_step_t<128>(sp, md, g, prescribed, err, s); break;
    case 256: launch_step_t<256>(sp, md, g, prescribed, err, s); break;
  }
}

template <int NR>
static void launch_observe_t(const SpeciesDev& sp, const MolDev& md, cudaStream_t s) {
  const size_t smem = mol_state_smem(NR, sp.nrot);
  cudaFuncSetAttribute(mol_observe_kernel<NR>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  mol_observe_kernel<NR><<<sp.nmol, FFTShape<NR>::THREADS, smem, s>>>(sp, md);
}

void launch_mol_observe(const SpeciesDev& sp, const MolDev& md, cudaStream_t s) {
  if (sp.nmol == 0) return;
  switch (sp.nr) {
    case 64: launch_observe_t<64>(sp, md, s); break;
    case 128: launch_observe_t<128>(sp, md, s); break;
    case 256: launch_observe_t<256>(sp, md, s); break;
  }
}

}  // namespace ms
