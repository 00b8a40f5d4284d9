// Internal device structures of the coupled Maxwell-Schroedinger library.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "ms.h"

namespace ms {

constexpr int kMaxMaterials = 16;
constexpr int kMaxSpecies = 8;
constexpr int kMaxJ = 16;
constexpr int kMaxRot = (kMaxJ + 1) * (kMaxJ + 1);  // 289 channels per surface
constexpr int kMaxCoupl = 6;                          // nonzeros of R^hat per row

// error bits latched in the device error word
enum : int {
  kErrNonFinite = 1,      // a molecule produced a non-finite population
  kErrCouplingSeries = 2, // |theta E'| too large for the coupling series
  kErrPrescribedRange = 4,
  kErrTimeout = 8,        // a bounded wait on an asynchronous copy gave up
  kErrLaunch = 16,        // a kernel could not be prepared (its tensor maps), so it did not run
};

// Incident wave parameters of one sim.
struct SrcParam {
  double E0;    // V/m
  double w;     // carrier, rad/s
  double fwhm;  // s: pulse envelope FWHM (MS_SRC_PULSE) or CW turn-on time (MS_SRC_CW)
  double t0;    // s
  int kind;     // MS_SRC_PULSE or MS_SRC_CW
};

// Incident field at the TF/SF plane at time t (the formulas of ms_grid_desc).
__host__ __device__ inline double incident_field(const SrcParam& p, double t) {
  const double u = t - p.t0;
  if (p.kind == 1) {
    double ramp = 1.0;
    if (t < p.fwhm) {
      const double r = sin(1.5707963267948966 * (t > 0.0 ? t : 0.0) / p.fwhm);
      ramp = r * r;
    }
    return p.E0 * ramp * cos(p.w * u);
  }
  const double x = u / p.fwhm;
  return p.E0 * exp(-2.772588722239781 * x * x) * cos(p.w * u);
}

// Per-material coefficients (constant memory).
struct MaterialCoef {
  float ce;     // dt / (eps0 eps_r dx): curl H -> E
  float cj;     // dt / (eps0 eps_r): Drude current -> E
  float cp;     // e a0 / (dx^3 eps0 eps_r): molecular dipole change (a.u.) -> E
  float alpha;  // Drude: J^{n+1/2} = alpha J^{n-1/2} + beta E^n
  float beta;
  int metal;    // 1 if wp > 0
};

// Field state and coefficients.
struct Grid {
  int nx, ny, nz, nsim;
  long long ncell_sim;   // nx*ny*nz
  float* E[3];
  float* H[3];
  const uint8_t* mat;
  MaterialCoef mc[kMaxMaterials];  // per material id
  float ch;              // dt / (mu0 dx): curl E -> H
  float ce_vac;          // dt / (eps0 dx): the incident line is vacuum
  int periodic_z;
  // Drude current, stored for z slab [jk0, jk1) only (metal cells)
  int jk0, jk1;
  float* J[3];
  // CPML: psi for k in [0, pml) (slab 0) and [nz-pml, nz) (slab 1)
  int pml;
  float* psiE[2];        // psi_Exz, psi_Eyz
  float* psiH[2];        // psi_Hxz, psi_Hyz
  const float4* cpml;    // per k: (bE, aE, bH, aH)
  // TF/SF source
  int ks;                // -1 = none
  int aux_len;
  float* auxE;           // [nsim][aux_len+1]
  float* auxH;           // [nsim][aux_len]
  const SrcParam* src;   // [nsim]
  double dt;
  // polarization current from molecules: CSR over the molecule z slab
  int mk0, mk1;          // slab [mk0, mk1) (empty when no molecules)
  const int* cell_off;   // [nsim*(mk1-mk0)*ny*nx + 1]
  const int* cell_mol;   // molecule ids sorted by cell
  const double* dmu;     // [nmol][3] lab dipole change of the last step (a.u.)
  long long* step;       // device step counter
  // spectral detection: running DFTs on z-planes, dt sum_n F(t_n) e^{i omega t_n}
  int ndet, nfreq;
  const int* det_k;      // [ndet] plane indices
  const double* omega;   // [nfreq] angular frequencies (rad/s)
  double2* dft;          // [nsim][ndet][nfreq][4][ny][nx]: Ex, Ey on plane k at t_{n+1};
                         // Hx, Hy averaged over z = k -+ 1/2 at t_{n+1/2}
};

// One species' device tables (all built on the host in FP64).
struct SpeciesDev {
  int nr, jmax, nrot;
  int par;                  // parity-reduced rows: ground even j, excited odd j
  int rows, rows_g;         // state rows per molecule, of which ground rows
  int nmol;                 // molecules of this species
  const int* mol;           // their global ids (sorted by species, then by id)
  float2* psi;              // state [nmol][rows][nr] (ground rows first), s = T^{-1/2} psi
  float2* d2;               // streaming form: scratch (T - 1) s, same layout
  float4* fld;              // streaming form: per molecule (theta E'_z, theta E'_x/2, theta E'_y/2, terms)
  int mixed;                // kinetic pass as the split-FP16 tensor-core GEMM (MS_PREC_MIXED_F16X3)
  const uint16_t* kpl;      // mixed: (K - I) strip as four FP16 planes (Re hi, Re lo, Im hi, Im lo), x 2^kpl_exp
  int kpl_exp;
  int path;                 // MS_MOL_FUSED or MS_MOL_STREAMING
  int kern, ch;             // plan: MS_KERN_* of the R-space pass, chunk width of the chunked kernel (0: its rule)
  int cps;                  // plan: grid of the persistent tiled kernel: resident CTAs per SM (> 0), 0 = as
                            // many as fit, -1 = one molecule per CTA
  // per (s, j, r): e^{-i V dtau} - 1 and e^{-i V dtau/2}
  const float2* vdelta;     // [2][jmax+1][nr]
  const float2* vhalf;      // [2][jmax+1][nr]
  const float2* kdelta;     // [nr] (e^{-i k^2 dtau / 2mu} - 1) / nr, natural k order
  const float2* khalf;      // [nr] e^{-i k^2 dtau / 4mu} / nr, for the psi = T^{1/2} s readout
  const float2* twiddle;    // [n2][n1]: exp(-2 pi i n1 k2 / nr)
  const float2* maskw;      // [nr]: (m, 1 - m^2)
  // the same three tables with each pair of radial points (2p, 2p + 1) as
  // (Re 2p, Re 2p+1), (Im 2p, Im 2p+1) (mask: (m, m), (1 - m^2, 1 - m^2)),
  // for the tiled kernel that holds two points a thread (MS_KERN_PAIR)
  const float2* vdelta_pp;
  const float2* vhalf_pp;
  const float2* maskw_pp;
  const float* r;           // [nr]
  double theta;             // d * dtau (d(R): its largest |d| times dtau)
  double dipole;            // d (e a0) (d(R): its largest |d|)
  const float* dipw;        // d(R) / max|d| at the grid points [nr], null for a constant dipole
  float dR;
  // frozen two-level molecules (MS_MODEL_BLOCH): Bloch vector per molecule
  int bloch;
  double* bloch_y;          // [nmol][3] (u, v, w), FP64
  double dtau;              // molecular step (a.u.)
  float bloch_w0;           // transition energy (a.u.)
  float bloch_g1, bloch_g2; // 1/T1, 1/T2 (a.u.), 0 = none
  double bloch_re;          // frozen bond length (a0), for the Eq. 8 readout
};

// One nonzero of an angular coupling row.
struct CouplEntry {
  int nbr;     // neighbour channel j^2 + j + m, -1 = unused
  float coef;
  int kind;
  int pad;
};

// Per-molecule data shared by all species.
struct MolDev {
  long long n;
  const int* cell;          // linear cell index including the sim offset (-1 unused)
  const float* rot;         // [n][9] molecule -> lab rotation, row-major
  double* mu;               // [n][3] lab dipole (a.u.)
  double* dmu;              // [n][3] change over the last step
  double* pop;              // [n][2] P_g, P_e
  double* absorbed;         // [n][2] cumulative absorbed norm
  double* Rnum;             // [n] Eq. 8 numerator (filled on readout)
  double* Rden;             // [n]
  // [n] rounding feedback of the wavepacket state: the relative norm change
  // sum(s'.e) / sum|s'|^2 that the last step's final FP32 rounding s' =
  // fl(s + D) introduced (e its exact TwoSum residual); the next step scales
  // its update by (1 + ncorr), which returns that norm, so rounding no longer
  // walks the norm.  Arithmetic error inside D is not compensated.
  float* ncorr;
  // prescribed drive
  const float* amp;         // [n][3]
  const float* wave;        // [nwave]
  long long nwave;
  const float* replay;      // replay drive [nwave][n][3] (lab V/m), else null
};

// Lab-frame field (V/m) driving molecule m during the current step: the
// replay samples, the prescribed amp x wave, or the components its cell owns
// on the grid (E^n, before this step's E update).
__device__ __forceinline__ void lab_field(const MolDev& md, const Grid& g, int prescribed, int m, float E[3],
                                          int* err) {
  const long long n = *g.step;
  if (prescribed) {
    const long long nn = n < md.nwave ? n : md.nwave - 1;
    if (n >= md.nwave) atomicOr(err, kErrPrescribedRange);
    if (md.replay) {
      const float* e = md.replay + (nn * md.n + m) * 3;
      E[0] = e[0];
      E[1] = e[1];
      E[2] = e[2];
    } else {
      const float wv = md.wave[nn];
      E[0] = md.amp[3 * (long long)m] * wv;
      E[1] = md.amp[3 * (long long)m + 1] * wv;
      E[2] = md.amp[3 * (long long)m + 2] * wv;
    }
  } else {
    const long long c = md.cell[m];
    E[0] = g.E[0][c];
    E[1] = g.E[1][c];
    E[2] = g.E[2][c];
  }
}

// launchers (yee.cu)
void launch_yee_h(const Grid& g, cudaStream_t s);
void launch_yee_e(const Grid& g, cudaStream_t s);

// launchers (mol.cu)
// one species' molecular step in two stages (see mol.cu); each returns the kernels it launched
int launch_mol_stage1(const SpeciesDev& sp, const MolDev& md, const Grid& g, int prescribed, int* err,
                      cudaStream_t s);
int launch_mol_stage2(const SpeciesDev& sp, const MolDev& md, const Grid& g, int prescribed, int* err,
                      cudaStream_t s);
void launch_mol_observe(const SpeciesDev& sp, const MolDev& md, cudaStream_t s);
// launchers (bloch.cu): the frozen two-level step and its Eq. 8 readout
int launch_bloch_step(const SpeciesDev& sp, const MolDev& md, const Grid& g, int prescribed, int* err,
                      cudaStream_t s);
void launch_bloch_observe(const SpeciesDev& sp, const MolDev& md, cudaStream_t s);
bool mol_step_supported(int nr, int nrot, int path);
// the driver's tensor-map encoder, which the tiled kernels need, is available
bool mol_tensor_maps_available();
// the (layout, kernel, chunk width, CTAs per SM) plans a species can run; returns how many
int mol_plan_candidates(const SpeciesDev& sp, int (*out)[4], int max);
cudaError_t upload_coupling_tables(const CouplEntry* rot, const CouplEntry* dip);
cudaError_t upload_triplet_tables(const CouplEntry* dip);
cudaError_t launch_wait_timeout_probe(int tries, int* flag, cudaStream_t s);
// mixed form of the kinetic pass: nr values it supports, the rows of the
// circulant strip of (K - I) and the byte offset of its element (row, q),
// q < 16, in the tensor cores' K-major layout
bool mol_mixed_supported(int nr);
int mixed_strip_rows(int nr);
int mixed_plane_offset(int row, int k, int nr);
void launch_step_counter(long long* step, cudaStream_t s);
void launch_dft(const Grid& g, cudaStream_t s);
// E^n at the cells of the listed molecules: out[k][3] for k < m
void launch_record_fields(const Grid& g, const int* cell, const long long* ids, int m, float* out,
                          cudaStream_t s);
cudaError_t launch_broadcast_row(float2* psi, const float2* row, int nr, size_t per, long long nmol,
                                 cudaStream_t s);

}  // namespace ms
