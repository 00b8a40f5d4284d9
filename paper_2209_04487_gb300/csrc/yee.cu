// Yee leap-frog kernels for Eq. 1 with the Drude current of Eq. 2, CPML
// along z, periodic x/y, TF/SF plane-wave source and the molecular
// polarization current (section "The domain decomposition methodology for
// FDTD"; coupling section for dP/dt).
//
// Both half steps are HBM-bound stencils: one thread per cell, x fastest so
// that a warp touches 128 contiguous bytes per component; the +-1 neighbours
// along y and z are re-read through L1/L2.
#include "ms_internal.cuh"

namespace ms {

struct CellIdx {
  int i, j, k, s;
};

__device__ __forceinline__ CellIdx decompose(long long c, const Grid& g) {
  CellIdx r;
  r.i = (int)(c % g.nx);
  long long t = c / g.nx;
  r.j = (int)(t % g.ny);
  t /= g.ny;
  r.k = (int)(t % g.nz);
  r.s = (int)(t / g.nz);
  return r;
}

__device__ __forceinline__ long long pml_index(const Grid& g, const CellIdx& q) {
  int slab = q.k < g.pml ? 0 : 1;
  int kk = q.k < g.pml ? q.k : q.k - (g.nz - g.pml);
  return (((long long)(q.s * 2 + slab) * g.pml + kk) * g.ny + q.j) * g.nx + q.i;
}

// H^{n-1/2} -> H^{n+1/2}
__global__ void __launch_bounds__(256) yee_h_kernel(Grid g) {
  const long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (c >= g.ncell_sim * g.nsim) return;
  const CellIdx q = decompose(c, g);
  const long long sxy = (long long)g.nx * g.ny;
  const long long cx = (q.i + 1 < g.nx) ? c + 1 : c - (g.nx - 1);
  const long long cy = (q.j + 1 < g.ny) ? c + g.nx : c - (long long)(g.ny - 1) * g.nx;
  long long cz = c + sxy;
  bool zero_top = false;
  if (q.k + 1 >= g.nz) {
    if (g.periodic_z) cz = c - (long long)(g.nz - 1) * sxy;
    else zero_top = true;  // perfect conductor above the top plane
  }
  const float* __restrict__ Ex = g.E[0];
  const float* __restrict__ Ey = g.E[1];
  const float* __restrict__ Ez = g.E[2];
  const float ex = Ex[c], ey = Ey[c], ez = Ez[c];
  const float ex_z = zero_top ? 0.f : Ex[cz];
  const float ey_z = zero_top ? 0.f : Ey[cz];
  float dEz_dy = Ez[cy] - ez;
  float dEy_dz = ey_z - ey;
  float dEx_dz = ex_z - ex;
  float dEz_dx = Ez[cx] - ez;
  float dEy_dx = Ey[cx] - ey;
  float dEx_dy = Ex[cy] - ex;
  if (g.pml > 0 && (q.k < g.pml || q.k >= g.nz - g.pml)) {
    const float4 co = g.cpml[q.k];  // (bE, aE, bH, aH); psi stored times dx
    const long long p = pml_index(g, q);
    const float px = co.z * g.psiH[0][p] + co.w * dEy_dz;
    const float py = co.z * g.psiH[1][p] + co.w * dEx_dz;
    g.psiH[0][p] = px;
    g.psiH[1][p] = py;
    dEy_dz += px;
    dEx_dz += py;
  }
  float hy_src = 0.f;
  if (q.k == g.ks - 1) hy_src = g.auxE[(long long)q.s * (g.aux_len + 1) + 2];
  g.H[0][c] -= g.ch * (dEz_dy - dEy_dz);
  g.H[1][c] = g.H[1][c] - g.ch * (dEx_dz - dEz_dx) + g.ch * hy_src;
  g.H[2][c] -= g.ch * (dEy_dx - dEx_dy);
}

// E^n -> E^{n+1}, with J_D^{n+1/2} and the molecular polarization change
__global__ void __launch_bounds__(256) yee_e_kernel(Grid g) {
  const long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (c >= g.ncell_sim * g.nsim) return;
  const CellIdx q = decompose(c, g);
  const long long sxy = (long long)g.nx * g.ny;
  const long long cx = (q.i > 0) ? c - 1 : c + (g.nx - 1);
  const long long cy = (q.j > 0) ? c - g.nx : c + (long long)(g.ny - 1) * g.nx;
  long long cz = c - sxy;
  bool zero_bot = false;
  if (q.k == 0) {
    if (g.periodic_z) cz = c + (long long)(g.nz - 1) * sxy;
    else zero_bot = true;
  }
  const float* __restrict__ Hx = g.H[0];
  const float* __restrict__ Hy = g.H[1];
  const float* __restrict__ Hz = g.H[2];
  const float hx = Hx[c], hy = Hy[c], hz = Hz[c];
  const float hx_z = zero_bot ? 0.f : Hx[cz];
  const float hy_z = zero_bot ? 0.f : Hy[cz];
  float dHz_dy = hz - Hz[cy];
  float dHy_dz = hy - hy_z;
  float dHx_dz = hx - hx_z;
  float dHz_dx = hz - Hz[cx];
  float dHy_dx = hy - Hy[cx];
  float dHx_dy = hx - Hx[cy];
  if (g.pml > 0 && (q.k < g.pml || q.k >= g.nz - g.pml)) {
    const float4 co = g.cpml[q.k];
    const long long p = pml_index(g, q);
    const float px = co.x * g.psiE[0][p] + co.y * dHy_dz;
    const float py = co.x * g.psiE[1][p] + co.y * dHx_dz;
    g.psiE[0][p] = px;
    g.psiE[1][p] = py;
    dHy_dz += px;
    dHx_dz += py;
  }
  float cxv = dHz_dy - dHy_dz;
  const float cyv = dHx_dz - dHz_dx;
  const float czv = dHy_dx - dHx_dy;
  if (q.k == g.ks) cxv += g.auxH[(long long)q.s * g.aux_len + 1];
  const MaterialCoef mc = g.mc[g.mat[c]];
  float ex = g.E[0][c], ey = g.E[1][c], ez = g.E[2][c];
  float jx = 0.f, jy = 0.f, jz = 0.f;
  if (mc.metal && q.k >= g.jk0 && q.k < g.jk1) {
    const long long jj =
        (((long long)q.s * (g.jk1 - g.jk0) + (q.k - g.jk0)) * g.ny + q.j) * g.nx + q.i;
    jx = mc.alpha * g.J[0][jj] + mc.beta * ex;
    jy = mc.alpha * g.J[1][jj] + mc.beta * ey;
    jz = mc.alpha * g.J[2][jj] + mc.beta * ez;
    g.J[0][jj] = jx;
    g.J[1][jj] = jy;
    g.J[2][jj] = jz;
  }
  ex += mc.ce * cxv - mc.cj * jx;
  ey += mc.ce * cyv - mc.cj * jy;
  ez += mc.ce * czv - mc.cj * jz;
  if (q.k >= g.mk0 && q.k < g.mk1) {
    const long long sl =
        (((long long)q.s * (g.mk1 - g.mk0) + (q.k - g.mk0)) * g.ny + q.j) * g.nx + q.i;
    const int b = g.cell_off[sl], e = g.cell_off[sl + 1];
    if (e > b) {
      double px = 0.0, py = 0.0, pz = 0.0;  // ensemble sum in FP64
      for (int t = b; t < e; ++t) {
        const int m = g.cell_mol[t];
        px += g.dmu[3 * (long long)m + 0];
        py += g.dmu[3 * (long long)m + 1];
        pz += g.dmu[3 * (long long)m + 2];
      }
      ex -= mc.cp * (float)px;
      ey -= mc.cp * (float)py;
      ez -= mc.cp * (float)pz;
    }
  }
  if (!g.periodic_z && q.k == 0) {
    ex = 0.f;  // tangential E on the bottom conductor
    ey = 0.f;
  }
  g.E[0][c] = ex;
  g.E[1][c] = ey;
  g.E[2][c] = ez;
}

// Incident line, H half step (one block per sim).  Node m of the line sits
// at z = (ks - 2 + m) dx; only nodes inside the numerical light cone of the
// source (m <= step + 2) can be non-zero, so only those are touched.
__global__ void aux_h_kernel(Grid g) {
  const int s = blockIdx.x;
  const long long n = *g.step;
  const int lim = (int)min((long long)g.aux_len, n + 4);
  float* E1 = g.auxE + (long long)s * (g.aux_len + 1);
  float* H1 = g.auxH + (long long)s * g.aux_len;
  for (int m = threadIdx.x; m < lim; m += blockDim.x) H1[m] -= g.ch * (E1[m + 1] - E1[m]);
}

__global__ void aux_e_kernel(Grid g) {
  const int s = blockIdx.x;
  const long long n = *g.step;
  const int lim = (int)min((long long)g.aux_len, n + 4);
  float* E1 = g.auxE + (long long)s * (g.aux_len + 1);
  const float* H1 = g.auxH + (long long)s * g.aux_len;
  const float ce = g.ce_vac;
  for (int m = 1 + threadIdx.x; m < lim; m += blockDim.x) E1[m] += ce * (0.f - (H1[m] - H1[m - 1]));
  if (threadIdx.x == 0) {
    E1[0] = (float)incident_field(g.src[s], (double)(n + 1) * g.dt);
  }
}

__global__ void step_counter_kernel(long long* step) { *step += 1; }

static unsigned blocks_for(long long n, int b) { return (unsigned)((n + b - 1) / b); }

void launch_yee_h(const Grid& g, cudaStream_t s) {
  const long long n = g.ncell_sim * g.nsim;
  yee_h_kernel<<<blocks_for(n, 256), 256, 0, s>>>(g);
}
void launch_yee_e(const Grid& g, cudaStream_t s) {
  const long long n = g.ncell_sim * g.nsim;
  yee_e_kernel<<<blocks_for(n, 256), 256, 0, s>>>(g);
}
void launch_aux_h(const Grid& g, cudaStream_t s) {
  if (g.ks >= 0) aux_h_kernel<<<g.nsim, 512, 0, s>>>(g);
}
void launch_aux_e(const Grid& g, cudaStream_t s) {
  if (g.ks >= 0) aux_e_kernel<<<g.nsim, 512, 0, s>>>(g);
}
// E^n at the cells of listed molecules (the coupled step's gather)
__global__ void record_fields_kernel(Grid g, const int* cell, const long long* ids, int m, float* out) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= m) return;
  const long long c = cell[ids[k]];
  out[3 * k] = g.E[0][c];
  out[3 * k + 1] = g.E[1][c];
  out[3 * k + 2] = g.E[2][c];
}
void launch_record_fields(const Grid& g, const int* cell, const long long* ids, int m, float* out,
                          cudaStream_t s) {
  record_fields_kernel<<<(m + 127) / 128, 128, 0, s>>>(g, cell, ids, m, out);
}
// Spectral detection: after the E update of step n (E^{n+1}, H^{n+1/2}),
// every cell of every detector plane adds dt F e^{i omega t} for each
// frequency: Ex, Ey of the plane at t_{n+1}; Hx, Hy averaged over the planes
// z = k - 1/2 and k + 1/2 (indices k - 1 and k) at t_{n+1/2}.  FP64.  A block
// covers 256 cells of one plane and kDftF frequencies.
constexpr int kDftF = 8;
__global__ void dft_kernel(Grid g, int nfc) {
  __shared__ double2 ph[2][kDftF];  // E and H phases of this block's frequencies, times dt
  const long long n = *g.step;
  const int d = blockIdx.y / nfc, f0 = (blockIdx.y % nfc) * kDftF, sim = blockIdx.z;
  const int nf = min(kDftF, g.nfreq - f0);
  if (threadIdx.x < nf) {
    double s1, c1, s2, c2;
    const double w = g.omega[f0 + threadIdx.x];
    sincos(w * (double)(n + 1) * g.dt, &s1, &c1);
    sincos(w * ((double)n + 0.5) * g.dt, &s2, &c2);
    ph[0][threadIdx.x] = make_double2(c1 * g.dt, s1 * g.dt);
    ph[1][threadIdx.x] = make_double2(c2 * g.dt, s2 * g.dt);
  }
  __syncthreads();
  const long long plane = (long long)g.ny * g.nx;
  const long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (q >= plane) return;
  const int k = g.det_k[d];
  const long long base = sim * g.ncell_sim;
  const long long ck = base + (long long)k * plane + q, cm = ck - plane;
  const double v[4] = {g.E[0][ck], g.E[1][ck], 0.5 * ((double)g.H[0][cm] + (double)g.H[0][ck]),
                       0.5 * ((double)g.H[1][cm] + (double)g.H[1][ck])};
  double2* acc = g.dft + (((long long)sim * g.ndet + d) * g.nfreq + f0) * 4 * plane + q;
  for (int f = 0; f < nf; ++f) {
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const double2 w = ph[c < 2 ? 0 : 1][f];
      double2* a = acc + ((long long)f * 4 + c) * plane;
      double2 x = *a;
      x.x = fma(v[c], w.x, x.x);
      x.y = fma(v[c], w.y, x.y);
      *a = x;
    }
  }
}
void launch_dft(const Grid& g, cudaStream_t s) {
  if (g.ndet <= 0) return;
  const long long plane = (long long)g.ny * g.nx;
  const int nfc = (g.nfreq + kDftF - 1) / kDftF;
  const dim3 grid((unsigned)((plane + 255) / 256), (unsigned)(g.ndet * nfc), (unsigned)g.nsim);
  dft_kernel<<<grid, 256, 0, s>>>(g, nfc);
}
void launch_step_counter(long long* step, cudaStream_t s) {
  step_counter_kernel<<<1, 1, 0, s>>>(step);
}

}  // namespace ms
