// Frozen two-level molecules (the scaling-experiments section, Fig. 5d):
// with the ro-vibrational degrees of freedom frozen, each molecule is a
// two-level emitter obeying the Bloch equations, advanced by one classical
// RK4 step per molecular step with the field held at E^n (the coupled
// step's order).  In atomic units, with W = 2 d (n . E) and n the molecular
// axis (the molecule frame's z axis in the lab):
//   du/dt =  w0 v - g2 u
//   dv/dt = -w0 u - W w - g2 v
//   dw/dt =  W v - g1 (w + 1)
// (u, v, w) = (2 Re rho_eg, 2 Im rho_eg, rho_ee - rho_gg); the dipole is
// d u along n.  One thread per molecule.  The Bloch vector stays in FP64 in
// HBM; the RK4 increment is formed in FP32 from the FP32-rounded vector and
// added in FP64, so its rounding scales with the increment (|W| dtau and
// w0 dtau are small), not with the unit-length vector.
#include "ms_internal.cuh"

namespace ms {

namespace {

struct Bv {
  float u, v, w;
};

__device__ __forceinline__ Bv bloch_rhs(Bv y, float w0, float W, float g1, float g2) {
  return {fmaf(w0, y.v, -g2 * y.u), fmaf(-w0, y.u, fmaf(-W, y.w, -g2 * y.v)), fmaf(W, y.v, -g1 * (y.w + 1.f))};
}
__device__ __forceinline__ Bv axpy(Bv y, float a, Bv k) {
  return {fmaf(a, k.u, y.u), fmaf(a, k.v, y.v), fmaf(a, k.w, y.w)};
}

__global__ void __launch_bounds__(128) mol_bloch_kernel(SpeciesDev sp, MolDev md, Grid g, int prescribed,
                                                        int* err) {
  const int lm = blockIdx.x * blockDim.x + threadIdx.x;
  if (lm >= sp.nmol) return;
  const int m = sp.mol[lm];
  float E[3];
  lab_field(md, g, prescribed, m, E, err);
  const float* O = md.rot + 9 * (long long)m;  // molecule -> lab, row-major: n = column 2
  const float nx = O[2], ny = O[5], nz = O[8];
  const float inv_fau = 1.0f / 5.14220674763e11f;
  const float W = 2.f * (float)sp.dipole * (nx * E[0] + ny * E[1] + nz * E[2]) * inv_fau;
  double* yp = sp.bloch_y + 3 * (long long)lm;
  const double u = yp[0], v = yp[1], w = yp[2];
  const float h = (float)sp.dtau, w0 = sp.bloch_w0, g1 = sp.bloch_g1, g2 = sp.bloch_g2;
  const Bv y = {(float)u, (float)v, (float)w};
  const Bv k1 = bloch_rhs(y, w0, W, g1, g2);
  const Bv k2 = bloch_rhs(axpy(y, 0.5f * h, k1), w0, W, g1, g2);
  const Bv k3 = bloch_rhs(axpy(y, 0.5f * h, k2), w0, W, g1, g2);
  const Bv k4 = bloch_rhs(axpy(y, h, k3), w0, W, g1, g2);
  const float c = h / 6.f;
  const double nu = u + (double)(c * (k1.u + 2.f * (k2.u + k3.u) + k4.u));
  const double nv = v + (double)(c * (k1.v + 2.f * (k2.v + k3.v) + k4.v));
  const double nw = w + (double)(c * (k1.w + 2.f * (k2.w + k3.w) + k4.w));
  if (!isfinite(nu) || !isfinite(nv) || !isfinite(nw)) atomicOr(err, kErrNonFinite);
  yp[0] = nu;
  yp[1] = nv;
  yp[2] = nw;
  md.pop[2 * (long long)m] = 0.5 * (1.0 - nw);
  md.pop[2 * (long long)m + 1] = 0.5 * (1.0 + nw);
  const double du = sp.dipole * nu;
  const double nl[3] = {du * nx, du * ny, du * nz};
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    md.dmu[3 * (long long)m + a] = nl[a] - md.mu[3 * (long long)m + a];
    md.mu[3 * (long long)m + a] = nl[a];
  }
}

// Eq. 8 with the bond frozen at r_e: numerator r_e P_e, denominator P_e
__global__ void __launch_bounds__(128) mol_bloch_observe_kernel(SpeciesDev sp, MolDev md) {
  const int lm = blockIdx.x * blockDim.x + threadIdx.x;
  if (lm >= sp.nmol) return;
  const int m = sp.mol[lm];
  const double pe = 0.5 * (1.0 + sp.bloch_y[3 * (long long)lm + 2]);
  md.Rnum[m] = sp.bloch_re * pe;
  md.Rden[m] = pe;
}

}  // namespace

int launch_bloch_step(const SpeciesDev& sp, const MolDev& md, const Grid& g, int prescribed, int* err,
                      cudaStream_t s) {
  if (sp.nmol == 0) return 0;
  mol_bloch_kernel<<<(sp.nmol + 127) / 128, 128, 0, s>>>(sp, md, g, prescribed, err);
  return 1;
}

void launch_bloch_observe(const SpeciesDev& sp, const MolDev& md, cudaStream_t s) {
  if (sp.nmol == 0) return;
  mol_bloch_observe_kernel<<<(sp.nmol + 127) / 128, 128, 0, s>>>(sp, md);
}

}  // namespace ms
