// Yee leap-frog kernels for Eq. 1 with the Drude current of Eq. 2, CPML
// along z, periodic x/y, TF/SF plane-wave source and the molecular
// polarization current (section "The domain decomposition methodology for
// FDTD"; coupling section for dP/dt).
//
// Both half steps are HBM-bound stencils: a thread marches along z through
// one (i, j) column, x fastest across the lanes so that a warp touches 128
// contiguous bytes per component; the z neighbour stays in registers, the x
// neighbour comes from the adjacent lane, the y neighbour through L1/L2.
#include "ms_internal.cuh"

namespace ms {

// The two half steps march along z: a block owns a tile of 32 x 8 columns
// (i, j) and kKz planes, one thread per column.  Each thread carries the
// plane it shares with the next (previous) cell of its column in registers,
// takes its x neighbour from the adjacent lane by a shuffle (the last lane of
// a warp, and the periodic wrap, load it), and reads its y neighbour through
// L1/L2.  Lanes outside the grid load a valid cell and store nothing.
constexpr int kTx = 32, kTy = 8, kKz = 8;

struct Tile {
  int i, j, s, k0, k1;
  bool in;
};

__device__ __forceinline__ Tile tile_of(const Grid& g, int b) {
  const int tx = (g.nx + kTx - 1) / kTx, ty = (g.ny + kTy - 1) / kTy, tz = (g.nz + kKz - 1) / kKz;
  Tile t;
  const int bx = b % tx;
  b /= tx;
  const int by = b % ty;
  b /= ty;
  const int bz = b % tz;
  t.s = b / tz;
  t.i = bx * kTx + (int)threadIdx.x;
  t.j = by * kTy + (int)threadIdx.y;
  t.k0 = bz * kKz;
  t.k1 = min(t.k0 + kKz, g.nz);
  t.in = t.i < g.nx && t.j < g.ny;
  return t;
}

static int yee_tiles(const Grid& g) {
  return ((g.nx + kTx - 1) / kTx) * ((g.ny + kTy - 1) / kTy) * ((g.nz + kKz - 1) / kKz) * g.nsim;
}

__device__ __forceinline__ long long pml_index(const Grid& g, int s, int k, int j, int i) {
  const int slab = k < g.pml ? 0 : 1;
  const int kk = k < g.pml ? k : k - (g.nz - g.pml);
  return (((long long)(s * 2 + slab) * g.pml + kk) * g.ny + j) * g.nx + i;
}

// Incident line, H half step (one block per sim).  Node m of the line sits
// at z = (ks - 2 + m) dx; only nodes inside the numerical light cone of the
// source (m <= step + 2) can be non-zero, so only those are touched.
__device__ void aux_h_block(const Grid& g, int s) {
  const long long n = *g.step;
  const int lim = (int)min((long long)g.aux_len, n + 4);
  float* E1 = g.auxE + (long long)s * (g.aux_len + 1);
  float* H1 = g.auxH + (long long)s * g.aux_len;
  const int t = threadIdx.y * kTx + threadIdx.x;
  for (int m = t; m < lim; m += kTx * kTy) H1[m] -= g.ch * (E1[m + 1] - E1[m]);
}

// Incident line, E half step, and the new source sample at its node 0.
__device__ void aux_e_block(const Grid& g, int s) {
  const long long n = *g.step;
  const int lim = (int)min((long long)g.aux_len, n + 4);
  float* E1 = g.auxE + (long long)s * (g.aux_len + 1);
  const float* H1 = g.auxH + (long long)s * g.aux_len;
  const float ce = g.ce_vac;
  const int t = threadIdx.y * kTx + threadIdx.x;
  for (int m = 1 + t; m < lim; m += kTx * kTy) E1[m] += ce * (0.f - (H1[m] - H1[m - 1]));
  if (t == 0) E1[0] = (float)incident_field(g.src[s], (double)(n + 1) * g.dt);
}

// H^{n-1/2} -> H^{n+1/2}.  Blocks past the tiles step the incident lines
// (they read only the lines; the tiles read only E and one line sample).
// The loads of plane k + 1 are issued before plane k is computed and stored,
// so every warp keeps two planes of loads in flight.
struct HPlane {
  float ez, ex_z, ey_z, ez_y, ex_y, ez_x, ey_x, h0, h1, h2;
};

__global__ void __launch_bounds__(kTx * kTy, 6) yee_h_kernel(Grid g, int ntiles) {
  if ((int)blockIdx.x >= ntiles) {
    aux_h_block(g, (int)blockIdx.x - ntiles);
    return;
  }
  const Tile t = tile_of(g, blockIdx.x);
  const int i = t.in ? t.i : 0, j = t.in ? t.j : 0;
  const int sxy = g.nx * g.ny;                                   // offsets within one sim (< 2^31 cells)
  const int dx = i + 1 < g.nx ? 1 : 1 - g.nx;                    // to (i + 1) mod nx
  const int dy = j + 1 < g.ny ? g.nx : -(g.ny - 1) * g.nx;       // to (j + 1) mod ny
  const int dzw = -(g.nz - 1) * sxy;                             // top plane -> bottom plane (periodic)
  const bool xsh = threadIdx.x + 1 < kTx && i + 1 < g.nx;        // the next lane holds i + 1
  const long long sb = (long long)t.s * g.ncell_sim;
  const float* __restrict__ Ex = g.E[0] + sb;
  const float* __restrict__ Ey = g.E[1] + sb;
  const float* __restrict__ Ez = g.E[2] + sb;
  float* __restrict__ H0 = g.H[0] + sb;
  float* __restrict__ H1 = g.H[1] + sb;
  float* __restrict__ H2 = g.H[2] + sb;
  const int c0 = t.k0 * sxy + j * g.nx + i;
  // plane k: E on k and k + 1 (zero above a conducting top), the y and x
  // neighbours (x only where no lane holds it), and H
  auto load = [&](int k, int c) {
    HPlane p;
    const bool top = k + 1 >= g.nz, zero_top = top && !g.periodic_z;
    const int cz = c + (top ? dzw : sxy);
    p.ez = Ez[c];
    p.ex_z = zero_top ? 0.f : Ex[cz];
    p.ey_z = zero_top ? 0.f : Ey[cz];
    p.ez_y = Ez[c + dy];
    p.ex_y = Ex[c + dy];
    p.ez_x = xsh ? 0.f : Ez[c + dx];
    p.ey_x = xsh ? 0.f : Ey[c + dx];
    p.h0 = H0[c];
    p.h1 = H1[c];
    p.h2 = H2[c];
    return p;
  };
  float ex = Ex[c0], ey = Ey[c0];  // plane k, carried from the previous iteration
  HPlane nx_ = load(t.k0, c0);
  int c = c0;
  for (int k = t.k0; k < t.k1; ++k, c += sxy) {
    const HPlane p = nx_;
    if (k + 1 < t.k1) nx_ = load(k + 1, c + sxy);
    const float ez_n = __shfl_down_sync(0xffffffffu, p.ez, 1);
    const float ey_n = __shfl_down_sync(0xffffffffu, ey, 1);
    const float ez_x = xsh ? ez_n : p.ez_x;
    const float ey_x = xsh ? ey_n : p.ey_x;
    float dEz_dy = p.ez_y - p.ez;
    float dEy_dz = p.ey_z - ey;
    float dEx_dz = p.ex_z - ex;
    const float dEz_dx = ez_x - p.ez;
    const float dEy_dx = ey_x - ey;
    const float dEx_dy = p.ex_y - ex;
    if (g.pml > 0 && (k < g.pml || k >= g.nz - g.pml)) {
      const float4 co = g.cpml[k];  // (bE, aE, bH, aH); psi stored times dx
      const long long q = pml_index(g, t.s, k, j, i);
      const float px = co.z * g.psiH[0][q] + co.w * dEy_dz;
      const float py = co.z * g.psiH[1][q] + co.w * dEx_dz;
      if (t.in) {
        g.psiH[0][q] = px;
        g.psiH[1][q] = py;
      }
      dEy_dz += px;
      dEx_dz += py;
    }
    float hy_src = 0.f;
    if (k == g.ks - 1) hy_src = g.auxE[(long long)t.s * (g.aux_len + 1) + 2];
    if (t.in) {
      H0[c] = p.h0 - g.ch * (dEz_dy - dEy_dz);
      H1[c] = p.h1 - g.ch * (dEx_dz - dEz_dx) + g.ch * hy_src;
      H2[c] = p.h2 - g.ch * (dEy_dx - dEx_dy);
    }
    ex = p.ex_z;
    ey = p.ey_z;
  }
}

// E^n -> E^{n+1}, with J_D^{n+1/2} and the molecular polarization change.
// Blocks past the tiles step the incident lines and set the new source
// sample (they read only the lines' H; the tiles read one H sample).
// Pipelined over the planes as the H half step.
struct EPlane {
  float hx, hy, hz, hz_y, hx_y, hz_x, hy_x, e0, e1, e2;
  int mat;
};

__global__ void __launch_bounds__(kTx * kTy, 5) yee_e_kernel(Grid g, int ntiles) {
  if ((int)blockIdx.x >= ntiles) {
    aux_e_block(g, (int)blockIdx.x - ntiles);
    return;
  }
  const Tile t = tile_of(g, blockIdx.x);
  const int i = t.in ? t.i : 0, j = t.in ? t.j : 0;
  const int sxy = g.nx * g.ny;                               // offsets within one sim (< 2^31 cells)
  const int dx = i > 0 ? 1 : 1 - g.nx;                       // from (i - 1) mod nx
  const int dy = j > 0 ? g.nx : -(g.ny - 1) * g.nx;          // from (j - 1) mod ny
  const bool xsh = threadIdx.x > 0 && i > 0;                 // the previous lane holds i - 1
  const long long sb = (long long)t.s * g.ncell_sim;
  const float* __restrict__ Hx = g.H[0] + sb;
  const float* __restrict__ Hy = g.H[1] + sb;
  const float* __restrict__ Hz = g.H[2] + sb;
  float* __restrict__ E0 = g.E[0] + sb;
  float* __restrict__ E1 = g.E[1] + sb;
  float* __restrict__ E2 = g.E[2] + sb;
  const uint8_t* __restrict__ mat = g.mat + sb;
  const int c0 = t.k0 * sxy + j * g.nx + i;
  auto load = [&](int c) {
    EPlane p;
    p.hx = Hx[c];
    p.hy = Hy[c];
    p.hz = Hz[c];
    p.hz_y = Hz[c - dy];
    p.hx_y = Hx[c - dy];
    p.hz_x = xsh ? 0.f : Hz[c - dx];
    p.hy_x = xsh ? 0.f : Hy[c - dx];
    p.e0 = E0[c];
    p.e1 = E1[c];
    p.e2 = E2[c];
    p.mat = mat[c];
    return p;
  };
  // plane k - 1, carried from the previous iteration
  float hx_m = 0.f, hy_m = 0.f;
  if (t.k0 > 0) {
    hx_m = Hx[c0 - sxy];
    hy_m = Hy[c0 - sxy];
  } else if (g.periodic_z) {
    hx_m = Hx[c0 + (g.nz - 1) * sxy];
    hy_m = Hy[c0 + (g.nz - 1) * sxy];
  }  // else: perfect conductor below the bottom plane
  EPlane nx_ = load(c0);
  int c = c0;
  for (int k = t.k0; k < t.k1; ++k, c += sxy) {
    const EPlane p = nx_;
    if (k + 1 < t.k1) nx_ = load(c + sxy);
    const float hz_n = __shfl_up_sync(0xffffffffu, p.hz, 1);
    const float hy_n = __shfl_up_sync(0xffffffffu, p.hy, 1);
    const float hz_x = xsh ? hz_n : p.hz_x;
    const float hy_x = xsh ? hy_n : p.hy_x;
    float dHz_dy = p.hz - p.hz_y;
    float dHy_dz = p.hy - hy_m;
    float dHx_dz = p.hx - hx_m;
    const float dHz_dx = p.hz - hz_x;
    const float dHy_dx = p.hy - hy_x;
    const float dHx_dy = p.hx - p.hx_y;
    hx_m = p.hx;
    hy_m = p.hy;
    if (g.pml > 0 && (k < g.pml || k >= g.nz - g.pml)) {
      const float4 co = g.cpml[k];
      const long long q = pml_index(g, t.s, k, j, i);
      const float px = co.x * g.psiE[0][q] + co.y * dHy_dz;
      const float py = co.x * g.psiE[1][q] + co.y * dHx_dz;
      if (t.in) {
        g.psiE[0][q] = px;
        g.psiE[1][q] = py;
      }
      dHy_dz += px;
      dHx_dz += py;
    }
    float cxv = dHz_dy - dHy_dz;
    const float cyv = dHx_dz - dHz_dx;
    const float czv = dHy_dx - dHx_dy;
    if (k == g.ks) cxv += g.auxH[(long long)t.s * g.aux_len + 1];
    if (t.in) {
      const MaterialCoef mc = g.mc[p.mat];
      float ex = p.e0, ey = p.e1, ez = p.e2;
      float jx = 0.f, jy = 0.f, jz = 0.f;
      if (mc.metal && k >= g.jk0 && k < g.jk1) {
        const long long jj = (((long long)t.s * (g.jk1 - g.jk0) + (k - g.jk0)) * g.ny + j) * g.nx + i;
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
      if (k >= g.mk0 && k < g.mk1) {
        const long long sl = (((long long)t.s * (g.mk1 - g.mk0) + (k - g.mk0)) * g.ny + j) * g.nx + i;
        const int b = g.cell_off[sl], e = g.cell_off[sl + 1];
        if (e > b) {
          double px = 0.0, py = 0.0, pz = 0.0;  // ensemble sum in FP64
          for (int q = b; q < e; ++q) {
            const int m = g.cell_mol[q];
            px += g.dmu[3 * (long long)m + 0];
            py += g.dmu[3 * (long long)m + 1];
            pz += g.dmu[3 * (long long)m + 2];
          }
          ex -= mc.cp * (float)px;
          ey -= mc.cp * (float)py;
          ez -= mc.cp * (float)pz;
        }
      }
      if (!g.periodic_z && k == 0) {
        ex = 0.f;  // tangential E on the bottom conductor
        ey = 0.f;
      }
      E0[c] = ex;
      E1[c] = ey;
      E2[c] = ez;
    }
  }
}

__global__ void step_counter_kernel(long long* step) { *step += 1; }


void launch_yee_h(const Grid& g, cudaStream_t s) {
  const int nt = yee_tiles(g);
  yee_h_kernel<<<nt + (g.ks >= 0 ? g.nsim : 0), dim3(kTx, kTy), 0, s>>>(g, nt);
}
void launch_yee_e(const Grid& g, cudaStream_t s) {
  const int nt = yee_tiles(g);
  yee_e_kernel<<<nt + (g.ks >= 0 ? g.nsim : 0), dim3(kTx, kTy), 0, s>>>(g, nt);
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
