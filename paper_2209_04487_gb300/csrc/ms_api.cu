// C ABI of the coupled Maxwell-Schroedinger library: validation, FP64 table
// construction on the host, device allocation, the step sequence and reads.
#include <cuda_runtime.h>

#include <algorithm>
#include <mutex>
#include <cmath>
#include <complex>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "ms.h"
#include "ms_internal.cuh"

namespace {

using cplx = std::complex<double>;

// CODATA 2018
constexpr double kC0 = 299792458.0;
constexpr double kMu0 = 1.25663706212e-6;
constexpr double kEps0 = 8.8541878128e-12;
constexpr double kHbarEVs = 6.582119569e-16;
constexpr double kTau = 2.4188843265857e-17;  // atomic unit of time, s
constexpr double kHartreeEV = 27.211386245988;  // atomic unit of energy, eV
constexpr double kEA0 = 8.4783536255e-30;     // atomic unit of dipole, C m
constexpr double kPi = 3.14159265358979323846;

// CPML grading (Roden-Gedney form, kappa = 1)
constexpr int kCpmlOrder = 3;
constexpr double kCpmlAlphaMax = 0.05;  // S/m
// incident line length (cells): exact for runs of up to ~4x this many steps
constexpr int kAuxLen = 32768;

// e^{i a} - 1 without cancellation
cplx expm1i(double a) {
  const double sh = std::sin(0.5 * a);
  return cplx(-2.0 * sh * sh, std::sin(a));
}

float2 f2(cplx z) { return make_float2((float)z.real(), (float)z.imag()); }

float4 hilo(cplx z) {
  const float ch = (float)z.real(), sh = (float)z.imag();
  return make_float4(ch, sh, (float)(z.real() - (double)ch), (float)(z.imag() - (double)sh));
}

struct Alloc {
  void* (*fn)(size_t, void*) = nullptr;
  void (*fr)(void*, void*) = nullptr;
  void* ctx = nullptr;
};

}  // namespace

constexpr int kMaxMolBatches = 16;  // runs per species of the pipelined molecular step

struct ms_sim {
  Alloc al;
  std::vector<void*> blocks;
  size_t bytes = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  int drive = MS_DRIVE_FDTD;
  int nspecies = 0;
  int64_t nmol = 0;
  int64_t steps = 0;
  int64_t nwave = 0;
  int nsub = 1;         // molecular step every nsub field steps
  // step replay from a CUDA graph of gsteps steps starting at phase 0
  bool graphs = true;
  cudaGraphExec_t gexec = nullptr;
  int gsteps = 0;
  bool gdirty = true;   // kernel arguments changed since the capture
  int src_kind = 0;     // MS_SRC_PULSE or MS_SRC_CW
  double dx = 0.0;      // cell size (m)
  ms::Grid g{};
  ms::MolDev md{};
  ms::SpeciesDev sp[ms::kMaxSpecies]{};
  int* d_err = nullptr;
  long long* d_step = nullptr;
  // device address of the library's fixed scratch array (ms_step_noalloc),
  // looked up at create with the handle's device current; null if that failed
  float2* noalloc_base = nullptr;
  std::vector<double> pop_init;  // create only: populations at t = 0, uploaded in one copy
  // phase timing
  bool timing = false;
  std::vector<cudaEvent_t> events;   // 4 per timed step
  int64_t timed_steps = 0, launches = 0;
  // pipelined molecular step (ms_set_mol_batches): runs per streaming species,
  // the second stream the R-space passes run on, and the events that order them
  int batches = 0;
  cudaStream_t stream2 = nullptr;
  std::vector<cudaEvent_t> bev;

  void* alloc(size_t n) {
    if (n == 0) n = 16;
    void* p = nullptr;
    if (al.fn) {
      p = al.fn(n, al.ctx);
    } else if (cudaMalloc(&p, n) != cudaSuccess) {
      cudaGetLastError();
      p = nullptr;
    }
    if (p) {
      blocks.push_back(p);
      bytes += n;
    }
    return p;
  }
  void release() {
    if (stream) cudaStreamSynchronize(stream);
    if (gexec) cudaGraphExecDestroy(gexec);
    gexec = nullptr;
    for (cudaEvent_t e : events) cudaEventDestroy(e);
    events.clear();
    if (stream2) cudaStreamSynchronize(stream2);
    for (cudaEvent_t e : bev) cudaEventDestroy(e);
    bev.clear();
    if (stream2) cudaStreamDestroy(stream2);
    stream2 = nullptr;
    for (void* p : blocks) {
      if (al.fr) al.fr(p, al.ctx);
      else cudaFree(p);
    }
    blocks.clear();
    if (own_stream && stream) cudaStreamDestroy(stream);
    stream = nullptr;
  }
};

namespace {

template <class T>
ms_status upload(ms_sim* s, T** dst, const T* src, size_t n) {
  void* p = s->alloc(n * sizeof(T));
  if (!p) return MS_ENOMEM;
  *dst = (T*)p;
  if (src && n && cudaMemcpyAsync(p, src, n * sizeof(T), cudaMemcpyHostToDevice, s->stream) != cudaSuccess)
    return MS_ECUDA;
  return MS_OK;
}

template <class T>
ms_status zeros(ms_sim* s, T** dst, size_t n) {
  void* p = s->alloc(n * sizeof(T));
  if (!p) return MS_ENOMEM;
  *dst = (T*)p;
  if (cudaMemsetAsync(p, 0, n * sizeof(T), s->stream) != cudaSuccess) return MS_ECUDA;
  return MS_OK;
}

#define MS_TRY(x)                      \
  do {                                 \
    const ms_status _st = (x);         \
    if (_st != MS_OK) return _st;      \
  } while (0)

// ---- Fourier-grid Hamiltonian ground state (Marston-Balint-Kurti), by
// inverse iteration with a Cholesky factorisation of H - sigma I, sigma
// below the spectrum.
bool fgh_ground_state(int n, double dR, double mass, const std::vector<double>& U,
                      std::vector<double>& psi) {
  std::vector<double> H((size_t)n * n, 0.0);
  for (int a = 0; a < n; ++a)
    for (int b = 0; b < n; ++b) {
      double t = 0.0;
      for (int p = -n / 2; p < n - n / 2; ++p) {
        const double k = 2.0 * kPi * p / (n * dR);
        t += k * k / (2.0 * mass) * std::cos(k * (a - b) * dR);
      }
      H[(size_t)a * n + b] = t / n;
    }
  double umin = U[0];
  for (int a = 0; a < n; ++a) {
    H[(size_t)a * n + a] += U[a];
    umin = std::min(umin, U[a]);
  }
  const double sigma = umin - 1e-3 * std::max(1.0, std::fabs(umin));
  for (int a = 0; a < n; ++a) H[(size_t)a * n + a] -= sigma;
  // Cholesky H = L L^T (lower, in place)
  for (int j = 0; j < n; ++j) {
    double d = H[(size_t)j * n + j];
    for (int k = 0; k < j; ++k) d -= H[(size_t)j * n + k] * H[(size_t)j * n + k];
    if (d <= 0.0) return false;
    d = std::sqrt(d);
    H[(size_t)j * n + j] = d;
    for (int i = j + 1; i < n; ++i) {
      double v = H[(size_t)i * n + j];
      for (int k = 0; k < j; ++k) v -= H[(size_t)i * n + k] * H[(size_t)j * n + k];
      H[(size_t)i * n + j] = v / d;
    }
  }
  std::vector<double> x(n, 1.0), y(n);
  for (int it = 0; it < 400; ++it) {
    for (int i = 0; i < n; ++i) {  // L y = x
      double v = x[i];
      for (int k = 0; k < i; ++k) v -= H[(size_t)i * n + k] * y[k];
      y[i] = v / H[(size_t)i * n + i];
    }
    for (int i = n - 1; i >= 0; --i) {  // L^T x = y
      double v = y[i];
      for (int k = i + 1; k < n; ++k) v -= H[(size_t)k * n + i] * x[k];
      x[i] = v / H[(size_t)i * n + i];
    }
    double nn = 0.0;
    for (double v : x) nn += v * v;
    nn = std::sqrt(nn);
    for (double& v : x) v /= nn;
  }
  int imax = 0;
  for (int i = 1; i < n; ++i)
    if (std::fabs(x[i]) > std::fabs(x[imax])) imax = i;
  const double sgn = x[imax] < 0 ? -1.0 : 1.0;
  double nrm = 0.0;
  for (double v : x) nrm += v * v * dR;
  nrm = std::sqrt(nrm);
  psi.resize(n);
  for (int i = 0; i < n; ++i) psi[i] = sgn * x[i] / nrm;
  return true;
}

int channel(int j, int m) { return j * j + j + m; }

// Angular matrix elements between complex spherical harmonics (Condon-
// Shortley): cos(t) couples (j,m)-(j+1,m) with a(j,m); sin(t)e^{ip} takes
// (j,m) to (j+1,m+1) with b(j,m) and to (j-1,m+1) with c(j,m).
double ang_a(int j, int m) { return std::sqrt(((j + 1.0) * (j + 1) - m * m) / ((2.0 * j + 1) * (2.0 * j + 3))); }
double ang_b(int j, int m) { return -std::sqrt((j + m + 1.0) * (j + m + 2) / ((2.0 * j + 1) * (2.0 * j + 3))); }
double ang_c(int j, int m) { return std::sqrt((j - m) * (j - m - 1.0) / ((2.0 * j - 1) * (2.0 * j + 1))); }

// Rows of E_perp X + E_z Z (the coupling in the frame where E'_y = 0) and of
// Z, S+, S- (for the dipole), for every channel up to kMaxJ.
ms_status upload_angular_tables() {
  const int J = ms::kMaxJ;
  auto valid = [J](int j, int m) { return j >= 0 && j <= J && m >= -j && m <= j; };
  std::vector<ms::CouplEntry> rot(ms::kMaxRot * ms::kMaxCoupl, ms::CouplEntry{-1, 0.f, 0, 0});
  std::vector<ms::CouplEntry> dip = rot;
  // fixed slots: rot 0-1 Z, 2-5 X; dip 0-1 Z, 2-3 S+, 4-5 S- (unused: nbr -1)
  for (int j = 0; j <= J; ++j)
    for (int m = -j; m <= j; ++m) {
      const size_t base = (size_t)channel(j, m) * ms::kMaxCoupl;
      auto put = [&](std::vector<ms::CouplEntry>& t, int slot, int jn, int mn, double coef) {
        if (!valid(jn, mn) || coef == 0.0) return;
        t[base + slot] = ms::CouplEntry{channel(jn, mn), (float)coef, slot, 0};
      };
      const double z0 = valid(j - 1, m) ? ang_a(j - 1, m) : 0.0, z1 = ang_a(j, m);
      // S+ row: from (j-1, m-1) and (j+1, m-1); S- row: from (j+1, m+1) and (j-1, m+1)
      const double p0 = valid(j - 1, m - 1) ? ang_b(j - 1, m - 1) : 0.0;
      const double p1 = valid(j + 1, m - 1) ? ang_c(j + 1, m - 1) : 0.0;
      const double q0 = ang_b(j, m);
      const double q1 = j >= 1 ? ang_c(j, m) : 0.0;
      put(rot, 0, j - 1, m, z0);
      put(rot, 1, j + 1, m, z1);
      put(rot, 2, j - 1, m - 1, 0.5 * p0);  // X = (S+ + S-)/2, four distinct channels
      put(rot, 3, j + 1, m - 1, 0.5 * p1);
      put(rot, 4, j + 1, m + 1, 0.5 * q0);
      put(rot, 5, j - 1, m + 1, 0.5 * q1);
      put(dip, 0, j - 1, m, z0);
      put(dip, 1, j + 1, m, z1);
      put(dip, 2, j - 1, m - 1, p0);
      put(dip, 3, j + 1, m - 1, p1);
      put(dip, 4, j + 1, m + 1, q0);
      put(dip, 5, j - 1, m + 1, q1);
    }
  if (ms::upload_coupling_tables(rot.data(), dip.data()) != cudaSuccess) return MS_ECUDA;
  return ms::upload_triplet_tables(dip.data()) == cudaSuccess ? MS_OK : MS_ECUDA;
}

// IEEE 754 binary16 of a finite double, rounded to nearest, ties to even
// (|v| below the largest finite half, 65504; callers scale into range).
uint16_t to_f16(double v) {
  const uint16_t sign = std::signbit(v) ? 0x8000u : 0u;
  const double a = std::fabs(v);
  if (a == 0.0) return sign;
  int e = 0;
  const double f = std::frexp(a, &e);  // a = f 2^e, f in [0.5, 1)
  int E = e - 1 + 15;                  // biased exponent of a normal half
  if (E >= 1) {
    int m = (int)std::nearbyint((2.0 * f - 1.0) * 1024.0);  // exact argument; ties to even
    if (m == 1024) {
      m = 0;
      ++E;
    }
    if (E >= 31) return (uint16_t)(sign | 0x7C00u);
    return (uint16_t)(sign | (E << 10) | m);
  }
  const int m = (int)std::nearbyint(std::ldexp(a, 24));  // subnormal: a = m 2^-24
  return (uint16_t)(sign | m);                          // m = 1024 is the smallest normal
}
double from_f16(uint16_t h) {
  const int E = (h >> 10) & 31, m = h & 1023;
  const double a = E == 0 ? std::ldexp((double)m, -24) : std::ldexp(1.0 + m / 1024.0, E - 15);
  return (h & 0x8000u) ? -a : a;
}

// (K - I) of the kinetic propagator for the mixed form, (K - I)[a][b] =
// (1/nr) sum_p (e^{-i k_p^2 dtau / 2 mu} - 1) e^{2 pi i p (a - b) / nr} (FP64),
// a circulant: stored as one 16-column strip T[i][q] = (K - I)[i - (nr - 16)][q]
// (indices mod nr) of 128 + nr - 16 rows, in four FP16 planes (Re hi, Re lo,
// Im hi, Im lo) in the tensor cores' K-major layout, scaled by 2^*exp2 so that
// its largest entry lies in [2^14, 2^15): hi + lo carries 22 bits of every
// entry.
std::vector<uint16_t> mixed_kinetic_planes(int nr, double dR, double dtau, double mu, int* exp2) {
  std::vector<cplx> kd(nr);
  double amax = 0.0;
  for (int dlt = 0; dlt < nr; ++dlt) {
    cplx acc = 0.0;
    for (int k = 0; k < nr; ++k) {
      const int p = k < nr / 2 ? k : k - nr;
      const double kk = 2.0 * kPi * p / (nr * dR);
      acc += expm1i(-kk * kk * dtau / (2.0 * mu)) * std::polar(1.0, 2.0 * kPi * p * dlt / nr);
    }
    kd[dlt] = acc / (double)nr;
    amax = std::max(amax, std::max(std::fabs(kd[dlt].real()), std::fabs(kd[dlt].imag())));
  }
  int ex = 0;
  std::frexp(amax > 0.0 ? amax : 1.0, &ex);
  *exp2 = 15 - ex;
  const int rows = ms::mixed_strip_rows(nr);
  const size_t plane = (size_t)rows * 16;  // elements
  std::vector<uint16_t> out(4 * plane, 0);
  for (int i = 0; i < rows; ++i)
    for (int q = 0; q < 16; ++q) {
      const int dlt = (((i - (nr - 16) - q) % nr) + nr) % nr;
      const double vr = std::ldexp(kd[dlt].real(), *exp2), vi = std::ldexp(kd[dlt].imag(), *exp2);
      const uint16_t rh = to_f16(vr), ih = to_f16(vi);
      const uint16_t rl = to_f16(vr - from_f16(rh)), il = to_f16(vi - from_f16(ih));
      const size_t off = (size_t)ms::mixed_plane_offset(i, q, nr) / 2;
      out[off] = rh;
      out[plane + off] = rl;
      out[2 * plane + off] = ih;
      out[3 * plane + off] = il;
    }
  return out;
}

// P_g, P_e of one species' molecules at t = 0, into the host copy of the
// population array that create uploads once every species is built
ms_status initial_populations(ms_sim* s, const std::vector<int>& ids, double pg) {
  for (size_t q = 0; q < ids.size(); ++q) {
    s->pop_init[2 * (size_t)ids[q]] = pg;
    s->pop_init[2 * (size_t)ids[q] + 1] = 0.0;
  }
  return MS_OK;
}

// Frozen two-level species (MS_MODEL_BLOCH): rates in atomic units, Bloch
// vectors at the ground state (0, 0, -1)
ms_status build_bloch_species(ms_sim* s, int si, const ms_species& d, double dt, const std::vector<int>& ids) {
  ms::SpeciesDev& sp = s->sp[si];
  sp.bloch = 1;
  sp.path = MS_MOL_FUSED;
  sp.nr = sp.jmax = sp.nrot = sp.rows = sp.rows_g = 0;
  sp.nmol = (int)ids.size();
  sp.dtau = dt / kTau;
  sp.dipole = d.dipole_ea0;
  sp.theta = d.dipole_ea0 * sp.dtau;
  sp.bloch_w0 = (float)(d.bloch_w0_eV / kHartreeEV);
  sp.bloch_g1 = d.bloch_T1_s > 0 ? (float)(kTau / d.bloch_T1_s) : 0.f;
  sp.bloch_g2 = d.bloch_T2_s > 0 ? (float)(kTau / d.bloch_T2_s) : 0.f;
  sp.bloch_re = d.morse_re;
  std::vector<double> y(3 * ids.size(), 0.0);
  for (size_t q = 0; q < ids.size(); ++q) y[3 * q + 2] = -1.0;
  MS_TRY(upload(s, &sp.bloch_y, y.data(), y.size()));
  MS_TRY(upload(s, (int**)&sp.mol, ids.data(), ids.size()));
  return initial_populations(s, ids, 1.0);
}

ms_status build_species(ms_sim* s, int si, const ms_species& d, double dt, const std::vector<int>& ids,
                        int path, bool mixed, bool par) {
  if (d.model == MS_MODEL_BLOCH) return build_bloch_species(s, si, d, dt, ids);
  ms::SpeciesDev& sp = s->sp[si];
  const int nr = d.nr, J = d.jmax, nrot = (J + 1) * (J + 1);
  // layout: the streaming form unless the caller asks for the fused one
  // MS_MOL_AUTO: the fused form where its point-resident kernel applies (FP32,
  // J <= 4, N_r = 128: one read and one write of the state per step), else
  // the streaming form
  const bool auto_fused = path == MS_MOL_AUTO && !mixed && d.jmax <= 4 && d.nr == 128;
  sp.path = (path == MS_MOL_FUSED || auto_fused) ? MS_MOL_FUSED : MS_MOL_STREAMING;
  sp.nr = nr;
  sp.jmax = J;
  sp.nrot = nrot;
  sp.nmol = (int)ids.size();
  sp.par = par ? 1 : 0;
  if (par) {  // ground rows: channels of even j; excited rows: odd j
    sp.rows_g = 0;
    sp.rows = 0;
    for (int j = 0; j <= J; ++j) {
      sp.rows += 2 * j + 1;
      if (j % 2 == 0) sp.rows_g += 2 * j + 1;
    }
  } else {
    sp.rows_g = nrot;
    sp.rows = 2 * nrot;
  }
  sp.mixed = mixed ? 1 : 0;
  sp.kpl = nullptr;
  const double dR = (d.rmax - d.rmin) / (nr - 1);
  const double dtau = dt / kTau;
  const double mu = d.mass_me;
  sp.dR = (float)dR;
  sp.theta = d.dipole_ea0 * dtau;
  sp.dipole = d.dipole_ea0;
  sp.dipw = nullptr;
  if (d.dipole_R) {  // d(R) = dipole * dipw[i]: the coupling's term count follows max |d|
    double dmax = 0.0;
    for (int i = 0; i < nr; ++i) dmax = std::max(dmax, std::fabs(d.dipole_R[i]));
    std::vector<float> w(nr);
    for (int i = 0; i < nr; ++i) w[i] = dmax > 0.0 ? (float)(d.dipole_R[i] / dmax) : 0.f;
    sp.dipole = dmax;
    sp.theta = dmax * dtau;
    MS_TRY(upload(s, (float**)&sp.dipw, w.data(), w.size()));
  }
  std::vector<double> r(nr), Ug(nr), Ue(nr);
  for (int i = 0; i < nr; ++i) {
    r[i] = d.rmin + i * dR;
    const double e = 1.0 - std::exp(-d.morse_a * (r[i] - d.morse_re));
    Ug[i] = d.morse_De * e * e - d.morse_De;
    Ue[i] = d.exc_A + d.exc_B * std::exp(-d.exc_beta * (r[i] - d.exc_rc));
  }
  // potential phases per (surface, j, r)
  std::vector<float2> vdelta((size_t)2 * (J + 1) * nr);
  std::vector<float2> vhalf((size_t)2 * (J + 1) * nr);
  for (int sf = 0; sf < 2; ++sf)
    for (int j = 0; j <= J; ++j)
      for (int i = 0; i < nr; ++i) {
        const double V = (sf == 0 ? Ug[i] : Ue[i]) + j * (j + 1) / (2.0 * mu * r[i] * r[i]);
        const size_t q = ((size_t)sf * (J + 1) + j) * nr + i;
        vdelta[q] = f2(expm1i(-V * dtau));
        const cplx h = std::polar(1.0, -0.5 * V * dtau);
        vhalf[q] = make_float2((float)h.real(), (float)h.imag());
      }
  // kinetic phases (natural DFT order) and four-step twiddles
  std::vector<float2> kph(nr), kphi(nr), tw(nr);
  for (int k = 0; k < nr; ++k) {
    const int p = k < nr / 2 ? k : k - nr;
    const double kk = 2.0 * kPi * p / (nr * dR);
    kph[k] = f2(expm1i(-kk * kk * dtau / (2.0 * mu)) / (double)nr);
    kphi[k] = f2(std::polar(1.0 / nr, -kk * kk * dtau / (4.0 * mu)));
  }
  const int N1 = nr == 64 ? 8 : 16, N2 = nr / N1;
  for (int n1 = 0; n1 < N1; ++n1)
    for (int k2 = 0; k2 < N2; ++k2) tw[k2 * N1 + n1] = f2(std::polar(1.0, -2.0 * kPi * n1 * k2 / nr));
  // absorber
  std::vector<float2> mw(nr);
  std::vector<float> rf(nr);
  for (int i = 0; i < nr; ++i) {
    double m = 1.0;
    if (d.absorber_r < d.rmax && r[i] > d.absorber_r) {
      const double x = (r[i] - d.absorber_r) / (d.rmax - d.absorber_r);
      m = std::pow(std::max(std::cos(0.5 * kPi * x), 0.0), d.absorber_power);
    }
    mw[i] = make_float2((float)m, (float)(1.0 - m * m));
    rf[i] = (float)r[i];
  }
  // initial state: v=0, j=0 Fourier-grid ground state, stored as s0 = T^{-1/2} psi0
  std::vector<double> psi0;
  if (!fgh_ground_state(nr, dR, mu, Ug, psi0)) return MS_EINVAL;
  std::vector<cplx> spec(nr), phi0(nr);
  for (int p = -nr / 2; p < nr - nr / 2; ++p) {
    const double k = 2.0 * kPi * p / (nr * dR);
    cplx acc = 0.0;
    for (int b = 0; b < nr; ++b) acc += psi0[b] * std::polar(1.0, -k * b * dR);
    spec[p + nr / 2] = acc * std::polar(1.0, +k * k * dtau / (4.0 * mu));
  }
  for (int a = 0; a < nr; ++a) {
    cplx acc = 0.0;
    for (int p = -nr / 2; p < nr - nr / 2; ++p) {
      const double k = 2.0 * kPi * p / (nr * dR);
      acc += spec[p + nr / 2] * std::polar(1.0, k * a * dR);
    }
    phi0[a] = acc / (double)nr;
  }
  const size_t per = (size_t)sp.rows * nr;
  std::vector<float2> row0(nr);
  for (int a = 0; a < nr; ++a) row0[a] = make_float2((float)phi0[a].real(), (float)phi0[a].imag());
  MS_TRY(zeros(s, &sp.psi, per * ids.size()));
  sp.d2 = nullptr;
  MS_TRY(zeros(s, &sp.fld, ids.size()));  // per-molecule frame-field records
  if (mixed) {
    const std::vector<uint16_t> kp = mixed_kinetic_planes(nr, dR, dtau, mu, &sp.kpl_exp);
    MS_TRY(upload(s, (uint16_t**)&sp.kpl, kp.data(), kp.size()));
  }
  if (sp.path == MS_MOL_STREAMING) MS_TRY(zeros(s, &sp.d2, per * ids.size()));
  float2* d_row0 = nullptr;
  MS_TRY(upload(s, &d_row0, row0.data(), row0.size()));
  if (ms::launch_broadcast_row(sp.psi, d_row0, nr, per, (long long)ids.size(), s->stream) != cudaSuccess)
    return MS_ECUDA;
  MS_TRY(upload(s, (float2**)&sp.vdelta, vdelta.data(), vdelta.size()));
  MS_TRY(upload(s, (float2**)&sp.vhalf, vhalf.data(), vhalf.size()));
  MS_TRY(upload(s, (float2**)&sp.kdelta, kph.data(), kph.size()));
  MS_TRY(upload(s, (float2**)&sp.khalf, kphi.data(), kphi.size()));
  MS_TRY(upload(s, (float2**)&sp.twiddle, tw.data(), tw.size()));
  MS_TRY(upload(s, (float2**)&sp.maskw, mw.data(), mw.size()));
  {  // pair layout of the potential and mask tables: (Re 2p, Re 2p+1, Im 2p, Im 2p+1) per point pair
    auto pairs = [nr](const std::vector<float2>& v) {
      std::vector<float2> o(v.size());
      for (size_t b = 0; b + 1 < v.size(); b += 2) {  // rows hold an even number of points
        o[b] = make_float2(v[b].x, v[b + 1].x);
        o[b + 1] = make_float2(v[b].y, v[b + 1].y);
      }
      (void)nr;
      return o;
    };
    const std::vector<float2> vdp = pairs(vdelta), vhp = pairs(vhalf), mwp = pairs(mw);
    MS_TRY(upload(s, (float2**)&sp.vdelta_pp, vdp.data(), vdp.size()));
    MS_TRY(upload(s, (float2**)&sp.vhalf_pp, vhp.data(), vhp.size()));
    MS_TRY(upload(s, (float2**)&sp.maskw_pp, mwp.data(), mwp.size()));
  }
  MS_TRY(upload(s, (float**)&sp.r, rf.data(), rf.size()));
  MS_TRY(upload(s, (int**)&sp.mol, ids.data(), ids.size()));
  // populations at t = 0
  double n0 = 0.0;
  for (double v : psi0) n0 += v * v * dR;
  return initial_populations(s, ids, n0);
}

// A plan switch to the streaming layout needs the (T - 1)s scratch.
ms_status ensure_scratch(ms_sim* s, ms::SpeciesDev& sp) {
  if (sp.d2 || sp.nmol == 0) return MS_OK;
  return zeros(s, &sp.d2, (size_t)sp.nmol * sp.rows * sp.nr);
}

// Device memory released before returning (the tuner's sandbox).
struct Scratch {
  ms_sim* s;
  std::vector<void*> p;
  void* get(size_t n) {
    void* q = nullptr;
    if (s->al.fn) q = s->al.fn(n ? n : 16, s->al.ctx);
    else if (cudaMalloc(&q, n ? n : 16) != cudaSuccess) {
      cudaGetLastError();
      q = nullptr;
    }
    if (q) p.push_back(q);
    return q;
  }
  ~Scratch() {
    cudaStreamSynchronize(s->stream);
    for (void* q : p) {
      if (s->al.fr) s->al.fr(q, s->al.ctx);
      else cudaFree(q);
    }
  }
};

// Measure every plan of species si on a sandbox copy of up to 2,048 of its
// molecules (own state, scratch, records and per-molecule arrays; the
// species' read-only tables are shared) under a prescribed field of 5e9 V/m
// along a seeded direction per molecule, and keep the fastest plan.
ms_status tune_species(ms_sim* s, int si) {
  ms::SpeciesDev& sp = s->sp[si];
  int cand[32][4];
  const int nc = ms::mol_plan_candidates(sp, cand, 32);
  if (nc < 2 || sp.nmol == 0) return MS_OK;
  const int nt = std::min(sp.nmol, 2048);
  const size_t per = (size_t)sp.rows * sp.nr;
  Scratch sc{s, {}};
  ms::SpeciesDev t = sp;
  ms::MolDev m = s->md;
  t.nmol = nt;
  t.psi = (float2*)sc.get(per * nt * sizeof(float2));
  t.d2 = (float2*)sc.get(per * nt * sizeof(float2));
  t.fld = (float4*)sc.get((size_t)nt * sizeof(float4));
  int* mol = (int*)sc.get((size_t)nt * sizeof(int));
  float* rot = (float*)sc.get((size_t)nt * 9 * sizeof(float));
  double* dbl = (double*)sc.get((size_t)nt * 14 * sizeof(double));  // mu, dmu, pop, absorbed, Rnum, Rden
  float* ncorr = (float*)sc.get((size_t)nt * sizeof(float));
  float* amp = (float*)sc.get((size_t)nt * 3 * sizeof(float));
  float* wave = (float*)sc.get(sizeof(float));
  long long* step = (long long*)sc.get(sizeof(long long));
  int* err = (int*)sc.get(sizeof(int));
  if (!t.psi || !t.d2 || !t.fld || !mol || !rot || !dbl || !ncorr || !amp || !wave || !step || !err)
    return MS_ENOMEM;
  // the first nt molecules of the species: state and rotations
  std::vector<int> ids(nt);
  if (cudaMemcpy(ids.data(), sp.mol, nt * sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return MS_ECUDA;
  std::vector<float> rh(9 * (size_t)nt);
  for (int k = 0; k < nt; ++k)
    if (cudaMemcpy(&rh[9 * (size_t)k], s->md.rot + 9 * (size_t)ids[k], 9 * sizeof(float),
                   cudaMemcpyDeviceToHost) != cudaSuccess)
      return MS_ECUDA;
  std::vector<int> iota(nt);
  std::vector<float> ah(3 * (size_t)nt);
  uint64_t x = 0x9E3779B97F4A7C15ull;  // splitmix64: a seeded direction per molecule
  for (int k = 0; k < nt; ++k) {
    iota[k] = k;
    double v[3], nn = 0.0;
    for (int c = 0; c < 3; ++c) {
      x += 0x9E3779B97F4A7C15ull;
      uint64_t z = x;
      z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
      z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
      z ^= z >> 31;
      v[c] = (double)(z >> 11) / 9007199254740992.0 - 0.5;
      nn += v[c] * v[c];
    }
    nn = std::sqrt(nn > 0 ? nn : 1.0);
    for (int c = 0; c < 3; ++c) ah[3 * (size_t)k + c] = (float)(5e9 * v[c] / nn);
  }
  const float one = 1.f;
  const long long zero = 0;
  if (cudaMemcpyAsync(t.psi, sp.psi, per * nt * sizeof(float2), cudaMemcpyDeviceToDevice, s->stream) != cudaSuccess ||
      cudaMemcpyAsync(mol, iota.data(), nt * sizeof(int), cudaMemcpyHostToDevice, s->stream) != cudaSuccess ||
      cudaMemcpyAsync(rot, rh.data(), rh.size() * sizeof(float), cudaMemcpyHostToDevice, s->stream) != cudaSuccess ||
      cudaMemcpyAsync(amp, ah.data(), ah.size() * sizeof(float), cudaMemcpyHostToDevice, s->stream) != cudaSuccess ||
      cudaMemcpyAsync(wave, &one, sizeof(float), cudaMemcpyHostToDevice, s->stream) != cudaSuccess ||
      cudaMemcpyAsync(step, &zero, sizeof(long long), cudaMemcpyHostToDevice, s->stream) != cudaSuccess ||
      cudaMemsetAsync(dbl, 0, (size_t)nt * 14 * sizeof(double), s->stream) != cudaSuccess ||
      cudaMemsetAsync(ncorr, 0, (size_t)nt * sizeof(float), s->stream) != cudaSuccess ||
      cudaMemsetAsync(err, 0, sizeof(int), s->stream) != cudaSuccess ||
      cudaStreamSynchronize(s->stream) != cudaSuccess)
    return MS_ECUDA;
  t.mol = mol;
  m.n = nt;
  m.cell = nullptr;
  m.rot = rot;
  m.mu = dbl;
  m.dmu = dbl + 3 * (size_t)nt;
  m.pop = dbl + 6 * (size_t)nt;
  m.absorbed = dbl + 8 * (size_t)nt;
  m.Rnum = dbl + 10 * (size_t)nt;
  m.Rden = dbl + 11 * (size_t)nt;
  m.ncorr = ncorr;
  m.amp = amp;
  m.wave = wave;
  m.nwave = 1;
  m.replay = nullptr;
  ms::Grid g = s->g;
  g.step = step;  // stays 0: the prescribed sample 0 every step
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    if (e0) cudaEventDestroy(e0);
    cudaGetLastError();
    return MS_ECUDA;
  }
  float best = 0.f;
  int pick = -1;
  for (int c = 0; c < nc; ++c) {
    t.path = cand[c][0];
    t.kern = cand[c][1];
    t.ch = cand[c][2];
    t.cps = cand[c][3];
    auto run = [&]() {
      ms::launch_mol_stage1(t, m, g, 1, err, s->stream);
      ms::launch_mol_stage2(t, m, g, 1, err, s->stream);
    };
    for (int w = 0; w < 2; ++w) run();
    cudaEventRecord(e0, s->stream);
    for (int r = 0; r < 5; ++r) run();
    cudaEventRecord(e1, s->stream);
    float ms_ = 0.f;
    if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms_, e0, e1) != cudaSuccess) {
      cudaEventDestroy(e0);
      cudaEventDestroy(e1);
      return MS_ECUDA;
    }
    if (pick < 0 || ms_ < best) {
      best = ms_;
      pick = c;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  int e = 0;
  if (cudaMemcpy(&e, err, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return MS_ECUDA;
  if (e != 0 || pick < 0) return MS_OK;  // a plan misbehaved in the sandbox: keep the static rule
  ms::SpeciesDev trial = sp;
  trial.path = cand[pick][0];
  if (trial.path == MS_MOL_STREAMING) MS_TRY(ensure_scratch(s, trial));
  sp = trial;
  sp.kern = cand[pick][1];
  sp.ch = cand[pick][2];
  sp.cps = cand[pick][3];
  return MS_OK;
}

ms_status create_impl(const ms_grid_desc* G, const ms_materials_desc* M, const ms_molecules_desc* D,
                      const ms_options* O, ms_sim* s) {
  const int nx = G->nx, ny = G->ny, nz = G->nz, nsim = G->nsim;
  const long long ncs = (long long)nx * ny * nz;
  const long long ncell = ncs * nsim;
  const double dx = G->dx_m, dt = G->dt_s;
  s->dx = dx;
  s->drive = O ? O->drive : MS_DRIVE_FDTD;
  s->nsub = O && O->mol_substeps > 1 ? O->mol_substeps : 1;
  s->graphs = !(O && O->step_graphs == MS_GRAPHS_OFF);
  s->src_kind = G->src_plane_z >= 0 ? G->src_kind : 0;
  s->nmol = D ? D->n_molecules : 0;
  s->nspecies = D ? D->n_species : 0;
  ms::Grid& g = s->g;
  g.nx = nx;
  g.ny = ny;
  g.nz = nz;
  g.nsim = nsim;
  g.ncell_sim = ncs;
  g.ch = (float)(dt / (kMu0 * dx));
  g.ce_vac = (float)(dt / (kEps0 * dx));
  g.periodic_z = G->bc_z == MS_BC_PERIODIC;
  g.dt = dt;
  MS_TRY(zeros(s, &g.step, 1));
  s->d_step = g.step;
  MS_TRY(zeros(s, &s->d_err, 1));
  MS_TRY(upload_angular_tables());
  // materials
  ms::MaterialCoef* mc = g.mc;
  for (int i = 0; i < M->n_materials; ++i) {
    const double er = M->eps_inf[i];
    mc[i].ce = (float)(dt / (kEps0 * er * dx));
    mc[i].cj = (float)(dt / (kEps0 * er));
    mc[i].cp = (float)(kEA0 / (dx * dx * dx * kEps0 * er));
    mc[i].metal = M->wp_eV[i] > 0;
    if (mc[i].metal) {
      const double wp = M->wp_eV[i] / kHbarEVs, ga = M->gamma_eV[i] / kHbarEVs;
      const double den = 1.0 + 0.5 * ga * dt;
      mc[i].alpha = (float)((1.0 - 0.5 * ga * dt) / den);
      mc[i].beta = (float)(kEps0 * wp * wp * dt / den);
    } else {
      mc[i].alpha = 1.f;
      mc[i].beta = 0.f;
    }
  }
  if (s->drive == MS_DRIVE_FDTD) {
    for (int c = 0; c < 3; ++c) {
      MS_TRY(zeros(s, &g.E[c], ncell));
      MS_TRY(zeros(s, &g.H[c], ncell));
    }
    MS_TRY(upload(s, (uint8_t**)&g.mat, M->material_id, ncell));
    // Drude slab: z range holding metal cells
    int jk0 = nz, jk1 = 0;
    for (long long c = 0; c < ncell; ++c)
      if (M->wp_eV[M->material_id[c]] > 0) {
        const int k = (int)((c / ((long long)nx * ny)) % nz);
        jk0 = std::min(jk0, k);
        jk1 = std::max(jk1, k + 1);
      }
    if (jk1 <= jk0) jk0 = jk1 = 0;
    g.jk0 = jk0;
    g.jk1 = jk1;
    const long long nj = (long long)nsim * (jk1 - jk0) * nx * ny;
    for (int c = 0; c < 3; ++c) MS_TRY(zeros(s, &g.J[c], nj > 0 ? nj : 1));
    // CPML
    g.pml = G->bc_z == MS_BC_PML ? G->pml_cells : 0;
    std::vector<float4> cpml(nz, make_float4(1.f, 0.f, 1.f, 0.f));
    if (g.pml > 0) {
      const double L = g.pml * dx;
      const double eta0 = std::sqrt(kMu0 / kEps0);
      const double smax = 0.8 * (kCpmlOrder + 1) / (eta0 * dx);
      auto prof = [&](double z, float* b, float* a) {
        const double rho = std::max(L - z, 0.0) + std::max(z - (nz * dx - L), 0.0);
        if (rho <= 0.0) {
          *b = 1.f;
          *a = 0.f;
          return;
        }
        const double sg = smax * std::pow(rho / L, kCpmlOrder);
        const double al = kCpmlAlphaMax * (1.0 - rho / L);
        const double bb = std::exp(-(sg + al) * dt / kEps0);
        *b = (float)bb;
        *a = (float)(sg > 0 ? sg / (sg + al) * (bb - 1.0) : 0.0);
      };
      for (int k = 0; k < nz; ++k) {
        prof(k * dx, &cpml[k].x, &cpml[k].y);
        prof((k + 0.5) * dx, &cpml[k].z, &cpml[k].w);
      }
      const long long np = (long long)nsim * 2 * g.pml * nx * ny;
      for (int c = 0; c < 2; ++c) {
        MS_TRY(zeros(s, &g.psiE[c], np));
        MS_TRY(zeros(s, &g.psiH[c], np));
      }
    }
    MS_TRY(upload(s, (float4**)&g.cpml, cpml.data(), cpml.size()));
    // TF/SF source
    g.ks = G->src_plane_z;
    g.aux_len = kAuxLen;
    if (g.ks >= 0) {
      std::vector<ms::SrcParam> sp(nsim);
      for (int q = 0; q < nsim; ++q) {
        sp[q].E0 = G->src[4 * q];
        sp[q].w = G->src[4 * q + 1] / kHbarEVs;
        sp[q].fwhm = G->src[4 * q + 2];
        sp[q].t0 = G->src[4 * q + 3];
        sp[q].kind = G->src_kind;
      }
      MS_TRY(upload(s, (ms::SrcParam**)&g.src, sp.data(), sp.size()));
      std::vector<float> aE((size_t)nsim * (kAuxLen + 1), 0.f);
      for (int q = 0; q < nsim; ++q) aE[(size_t)q * (kAuxLen + 1)] = (float)ms::incident_field(sp[q], 0.0);
      MS_TRY(upload(s, &g.auxE, aE.data(), aE.size()));
      MS_TRY(zeros(s, &g.auxH, (size_t)nsim * kAuxLen));
    }
  } else {
    g.ks = -1;
  }
  // molecules
  const long long n = s->nmol;
  ms::MolDev& md = s->md;
  md.n = n;
  std::vector<int> cell(n > 0 ? n : 1, -1);
  std::vector<float> rot(9 * (n > 0 ? n : 1), 0.f);
  int mk0 = nz, mk1 = 0;
  for (long long q = 0; q < n; ++q) {
    const int ci = (int)std::floor(D->pos_m[3 * q] / dx);
    const int cj = (int)std::floor(D->pos_m[3 * q + 1] / dx);
    const int ck = (int)std::floor(D->pos_m[3 * q + 2] / dx);
    const int sm = D->sim_id ? D->sim_id[q] : 0;
    cell[q] = (int)(((long long)sm * nz + ck) * ny * nx + (long long)cj * nx + ci);
    mk0 = std::min(mk0, ck);
    mk1 = std::max(mk1, ck + 1);
    double w = D->orient[4 * q], x = D->orient[4 * q + 1], y = D->orient[4 * q + 2], z = D->orient[4 * q + 3];
    const double nn = std::sqrt(w * w + x * x + y * y + z * z);
    w /= nn; x /= nn; y /= nn; z /= nn;
    const double R[9] = {1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y),
                         2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x),
                         2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)};
    for (int e = 0; e < 9; ++e) rot[9 * q + e] = (float)R[e];
  }
  if (n == 0) mk0 = mk1 = 0;
  g.mk0 = mk0;
  g.mk1 = mk1;
  MS_TRY(upload(s, (int**)&md.cell, cell.data(), cell.size()));
  MS_TRY(upload(s, (float**)&md.rot, rot.data(), rot.size()));
  const size_t nn1 = n > 0 ? n : 1;
  MS_TRY(zeros(s, &md.mu, 3 * nn1));
  MS_TRY(zeros(s, &md.dmu, 3 * nn1));
  MS_TRY(zeros(s, &md.pop, 2 * nn1));
  MS_TRY(zeros(s, &md.absorbed, 2 * nn1));
  MS_TRY(zeros(s, &md.Rnum, nn1));
  MS_TRY(zeros(s, &md.Rden, nn1));
  MS_TRY(zeros(s, &md.ncorr, nn1));
  g.dmu = md.dmu;
  if (s->drive == MS_DRIVE_FDTD && n > 0) {
    // CSR over the molecule slab: cells sorted, molecules of a cell in id order
    const long long nsl = (long long)nsim * (mk1 - mk0) * ny * nx;
    std::vector<int> off(nsl + 1, 0), lst(n);
    std::vector<long long> sl(n);
    for (long long q = 0; q < n; ++q) {
      const long long c = cell[q];
      const long long sm = c / ncs, rem = c % ncs;
      const long long k = rem / ((long long)nx * ny), ij = rem % ((long long)nx * ny);
      sl[q] = (sm * (mk1 - mk0) + (k - mk0)) * nx * ny + ij;
      off[sl[q] + 1]++;
    }
    for (long long c = 0; c < nsl; ++c) off[c + 1] += off[c];
    std::vector<int> fill(off.begin(), off.end() - 1);
    for (long long q = 0; q < n; ++q) lst[fill[sl[q]]++] = (int)q;
    MS_TRY(upload(s, (int**)&g.cell_off, off.data(), off.size()));
    MS_TRY(upload(s, (int**)&g.cell_mol, lst.data(), lst.size()));
  }
  // species
  s->pop_init.assign(2 * nn1, 0.0);
  for (int si = 0; si < s->nspecies; ++si) {
    std::vector<int> ids;
    for (long long q = 0; q < n; ++q)
      if (D->species_id[q] == si) ids.push_back((int)q);
    MS_TRY(build_species(s, si, D->species[si], dt * s->nsub, ids, O ? O->mol_path : MS_MOL_AUTO,
                         O && O->precision == MS_PREC_MIXED_F16X3, O && O->state_form == MS_STATE_PARITY));
  }
  if (cudaMemcpyAsync(md.pop, s->pop_init.data(), s->pop_init.size() * sizeof(double), cudaMemcpyHostToDevice,
                      s->stream) != cudaSuccess ||
      cudaStreamSynchronize(s->stream) != cudaSuccess)
    return MS_ECUDA;
  std::vector<double>().swap(s->pop_init);
  if (O && O->autotune == MS_TUNE_MEASURE)
    for (int si = 0; si < s->nspecies; ++si) MS_TRY(tune_species(s, si));
  return MS_OK;
}

ms_status validate(const ms_grid_desc* G, const ms_materials_desc* M, const ms_molecules_desc* D,
                   const ms_options* O) {
  if (!G || !M) return MS_EINVAL;
  if (G->nx <= 0 || G->ny <= 0 || G->nz <= 2 || G->nsim <= 0) return MS_EINVAL;
  if (!(G->dx_m > 0) || !(G->dt_s > 0)) return MS_EINVAL;
  if (G->dt_s > G->dx_m / (std::sqrt(3.0) * kC0)) return MS_EINVAL;
  const long long ncell = (long long)G->nx * G->ny * G->nz * G->nsim;
  if (ncell >= (1LL << 31)) return MS_EUNSUPPORTED;
  if (G->bc_z != MS_BC_PML && G->bc_z != MS_BC_PERIODIC) return MS_EINVAL;
  if (G->bc_z == MS_BC_PML && (G->pml_cells < 0 || 2 * G->pml_cells >= G->nz)) return MS_EINVAL;
  if (G->src_plane_z >= 0) {
    if (!G->src || G->bc_z != MS_BC_PML) return MS_EINVAL;
    if (G->src_kind != MS_SRC_PULSE && G->src_kind != MS_SRC_CW) return MS_EINVAL;
    if (G->src_plane_z < G->pml_cells + 2 || G->src_plane_z >= G->nz - G->pml_cells) return MS_EINVAL;
    for (int q = 0; q < G->nsim; ++q)
      if (!(G->src[4 * q + 2] > 0)) return MS_EINVAL;
  }
  if (M->n_materials <= 0 || M->n_materials > ms::kMaxMaterials || !M->eps_inf || !M->wp_eV ||
      !M->gamma_eV || !M->material_id)
    return MS_EINVAL;
  for (int i = 0; i < M->n_materials; ++i)
    if (!(M->eps_inf[i] > 0) || M->wp_eV[i] < 0 || M->gamma_eV[i] < 0) return MS_EINVAL;
  for (long long c = 0; c < ncell; ++c)
    if (M->material_id[c] >= M->n_materials) return MS_EINVAL;
  const int drive = O ? O->drive : MS_DRIVE_FDTD;
  if (drive != MS_DRIVE_FDTD && drive != MS_DRIVE_PRESCRIBED) return MS_EINVAL;
  if (O && O->precision != MS_PREC_FP32 && O->precision != MS_PREC_MIXED_F16X3) return MS_EINVAL;
  const bool mixed = O && O->precision == MS_PREC_MIXED_F16X3;
  if (O && (O->mol_substeps < 0 || O->mol_substeps > 65536)) return MS_EINVAL;
  if (O && ((O->alloc == nullptr) != (O->free == nullptr))) return MS_EINVAL;
  if (O && (O->mol_path < MS_MOL_AUTO || O->mol_path > MS_MOL_STREAMING)) return MS_EINVAL;
  if (O && O->state_form != MS_STATE_FULL && O->state_form != MS_STATE_PARITY) return MS_EINVAL;
  if (O && O->step_graphs != MS_GRAPHS_AUTO && O->step_graphs != MS_GRAPHS_OFF) return MS_EINVAL;
  if (O && O->autotune != MS_TUNE_OFF && O->autotune != MS_TUNE_MEASURE) return MS_EINVAL;
  const bool par = O && O->state_form == MS_STATE_PARITY;
  if (D && D->n_molecules > 0) {
    if (D->n_species <= 0 || D->n_species > ms::kMaxSpecies || !D->species || !D->species_id ||
        !D->pos_m || !D->orient)
      return MS_EINVAL;
    if (D->n_molecules >= (1LL << 31)) return MS_EUNSUPPORTED;
    for (int si = 0; si < D->n_species; ++si) {
      const ms_species& sp = D->species[si];
      if (sp.model == MS_MODEL_BLOCH) {  // frozen two-level emitter: its own parameters only
        if (!(sp.bloch_w0_eV >= 0) || !(sp.bloch_T1_s >= 0) || !(sp.bloch_T2_s >= 0) ||
            !std::isfinite(sp.bloch_w0_eV) || !std::isfinite(sp.bloch_T1_s) || !std::isfinite(sp.bloch_T2_s) ||
            !std::isfinite(sp.dipole_ea0) || !std::isfinite(sp.morse_re))
          return MS_EINVAL;
        continue;
      }
      if (sp.model != MS_MODEL_WAVEPACKET) return MS_EINVAL;
      if (sp.nr != 64 && sp.nr != 128 && sp.nr != 256) return MS_EUNSUPPORTED;
      if (sp.dipole_R) {  // R-dependent dipole: the point-resident kernels only
        for (int i = 0; i < sp.nr; ++i)
          if (!std::isfinite(sp.dipole_R[i])) return MS_EINVAL;
        const int path = O ? O->mol_path : MS_MOL_AUTO;
        if (sp.jmax > 4 || sp.nr == 256 || par || (path == MS_MOL_FUSED && sp.nr != 128)) return MS_EUNSUPPORTED;
      }
      if (sp.jmax < 0 || sp.jmax > ms::kMaxJ) return MS_EUNSUPPORTED;
      if (!(sp.rmax > sp.rmin) || !(sp.rmin > 0) || !(sp.mass_me > 0) || sp.absorber_power < 0)
        return MS_EINVAL;
      const int nrot = (sp.jmax + 1) * (sp.jmax + 1);
      const int path = O ? O->mol_path : MS_MOL_AUTO;
      if (path == MS_MOL_FUSED ? !ms::mol_step_supported(sp.nr, nrot, MS_MOL_FUSED)
                               : !ms::mol_step_supported(sp.nr, nrot, MS_MOL_STREAMING))
        return MS_EUNSUPPORTED;
      // the mixed kinetic pass: streaming form, radial grids of 64 or 128 points
      if (mixed && (path == MS_MOL_FUSED || !ms::mol_mixed_supported(sp.nr))) return MS_EUNSUPPORTED;
      // parity-reduced rows: the point-resident kernels (J <= 4; fused only at N_r = 128), and from
      // J = 5 on the two-points-a-thread tiled kernel (streaming layout, FP32 kinetic pass)
      if (par && sp.jmax <= 4 && path == MS_MOL_FUSED && sp.nr != 128) return MS_EUNSUPPORTED;
      if (par && sp.jmax >= 5 && (path == MS_MOL_FUSED || mixed || !ms::mol_tensor_maps_available()))
        return MS_EUNSUPPORTED;
    }
    for (long long q = 0; q < D->n_molecules; ++q) {
      const int si = D->species_id[q];
      if (si < 0 || si >= D->n_species) return MS_EINVAL;
      const int sm = D->sim_id ? D->sim_id[q] : 0;
      if (sm < 0 || sm >= G->nsim) return MS_EINVAL;
      const double* p = D->pos_m + 3 * q;
      const int ext[3] = {G->nx, G->ny, G->nz};
      for (int a = 0; a < 3; ++a) {
        const double c = std::floor(p[a] / G->dx_m);
        if (!(c >= 0) || c >= ext[a]) return MS_EINVAL;
      }
      const double* o = D->orient + 4 * q;
      const double nn = o[0] * o[0] + o[1] * o[1] + o[2] * o[2] + o[3] * o[3];
      if (!(nn > 1e-12) || !std::isfinite(nn)) return MS_EINVAL;
    }
  }
  return MS_OK;
}

}  // namespace

// ---- allocation-free stepping --------------------------------------------
// A fixed device array compiled into the library stands in for the per-
// species (T - 1)s scratch of the streaming form, one disjoint region per
// streaming species.  Every GPU that loads the library holds it until the
// process exits.  In host code `g_noalloc_scratch` is only a stand-in symbol:
// its device address is looked up once per device (with that device current,
// from ms_create) and passed to the kernels.
namespace {
constexpr size_t kNoAllocScratchBytes = 64ull << 20;  // 64 MiB
static __device__ __align__(256) float2 g_noalloc_scratch[kNoAllocScratchBytes / sizeof(float2)];

constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mutex;
float2* g_noalloc_addr[kMaxDevices] = {};

ms_status noalloc_scratch(float2** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return MS_ECUDA;
  std::lock_guard<std::mutex> lock(g_noalloc_mutex);
  if (!g_noalloc_addr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
      cudaGetLastError();
      return MS_ECUDA;
    }
    g_noalloc_addr[dev] = static_cast<float2*>(p);
  }
  *out = g_noalloc_addr[dev];
  return MS_OK;
}
}  // namespace

extern "C" {

const char* ms_status_string(ms_status s) {
  switch (s) {
    case MS_OK: return "ok";
    case MS_EINVAL: return "invalid argument";
    case MS_ENOMEM: return "device allocation failed";
    case MS_ECUDA: return "CUDA runtime error";
    case MS_ENUMERIC: return "non-finite value or coupling series out of range";
    case MS_ETIMEOUT: return "device wait timed out";
    case MS_EUNSUPPORTED: return "unsupported device or configuration";
    case MS_EIO: return "checkpoint file error";
  }
  return "unknown status";
}

ms_status ms_create(const ms_grid_desc* grid, const ms_materials_desc* materials,
                    const ms_molecules_desc* molecules, const ms_options* opts, ms_sim** out) {
  if (!out) return MS_EINVAL;
  *out = nullptr;
  const ms_status v = validate(grid, materials, molecules, opts);
  if (v != MS_OK) return v;
  int dev = 0;
  cudaDeviceProp prop;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaGetDeviceProperties(&prop, dev) != cudaSuccess) {
    cudaGetLastError();
    return MS_EUNSUPPORTED;
  }
  if (prop.major != 10 || prop.minor != 3) return MS_EUNSUPPORTED;
  ms_sim* s = new (std::nothrow) ms_sim();
  if (!s) return MS_ENOMEM;
  if (opts && opts->alloc) {
    s->al.fn = opts->alloc;
    s->al.fr = opts->free;
    s->al.ctx = opts->alloc_ctx;
  }
  if (opts && opts->stream) {
    s->stream = (cudaStream_t)opts->stream;
  } else {
    if (cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking) != cudaSuccess) {
      delete s;
      return MS_ECUDA;
    }
    s->own_stream = true;
  }
  const ms_status st = create_impl(grid, materials, molecules, opts, s);
  // the fixed scratch of ms_step_noalloc, looked up now so that the stepping
  // call only reads the pointer; a failure here only disables that call
  if (st == MS_OK && noalloc_scratch(&s->noalloc_base) != MS_OK) s->noalloc_base = nullptr;
  if (st != MS_OK) {
    cudaGetLastError();
    s->release();
    delete s;
    return st;
  }
  *out = s;
  return MS_OK;
}

static ms_status latched(ms_sim* s) {
  int e = 0;
  if (cudaMemcpyAsync(&e, s->d_err, sizeof(int), cudaMemcpyDeviceToHost, s->stream) != cudaSuccess)
    return MS_ECUDA;
  if (cudaStreamSynchronize(s->stream) != cudaSuccess) return MS_ECUDA;
  if (e & ms::kErrPrescribedRange) return MS_EINVAL;
  if (e & ms::kErrTimeout) return MS_ETIMEOUT;
  if (e & ms::kErrLaunch) return MS_ECUDA;
  return e ? MS_ENUMERIC : MS_OK;
}

static cudaEvent_t mark(ms_sim* s) {
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
  cudaEventRecord(e, s->stream);
  s->events.push_back(e);
  return e;
}

// One coupled step: H half step, the molecules (stage 1: field records and
// kinetic pass; stage 2: R-space pass, for every species), E half step.
// `scratch`, when set, gives each streaming species a d2 buffer that replaces
// its own (scratch[si], one disjoint region per species).
struct FieldRecorder {  // ms_record_local_fields: E^n of listed molecules, one row per step
  const long long* ids;
  int m;
  float* out;  // [steps][m][3], advanced by the caller
};

// The pipelined molecular step (ms_set_mol_batches): every streaming species'
// molecules in s->batches runs of consecutive molecules (other species: one
// run), ordered species by species.  Stage 1 (field records, kinetic pass) of
// run k + 1 is issued on the handle's stream right after that of run k; stage
// 2 (R-space pass) of run k waits for its stage 1 on the second stream.  The
// runs touch disjoint molecules, so stage 1 of one run may overlap stage 2 of
// the previous one; the handle's stream then waits for the last stage 2.
// Every molecule gets the same kernels on the same data: results do not
// depend on the batching.
static int pipelined_molecules(ms_sim* s, const ms::SpeciesDev* sp, int prescribed) {
  ms::SpeciesDev runs[ms::kMaxSpecies * kMaxMolBatches];
  int nrun = 0;
  for (int si = 0; si < s->nspecies; ++si) {
    const ms::SpeciesDev& a = sp[si];
    const int nb = a.path == MS_MOL_STREAMING && !a.bloch ? std::min(s->batches, std::max(a.nmol, 1)) : 1;
    const size_t per = (size_t)a.rows * a.nr;
    for (int b = 0; b < nb; ++b) {
      const int lo = (int)((long long)a.nmol * b / nb), hi = (int)((long long)a.nmol * (b + 1) / nb);
      ms::SpeciesDev r = a;
      r.nmol = hi - lo;
      r.mol = a.mol + lo;
      r.psi = a.psi + per * lo;
      if (a.d2) r.d2 = a.d2 + per * lo;
      r.fld = a.fld + lo;
      if (a.bloch_y) r.bloch_y = a.bloch_y + 3 * (size_t)lo;
      runs[nrun++] = r;
    }
  }
  int launched = 0;
  for (int k = 0; k < nrun; ++k) {
    launched += ms::launch_mol_stage1(runs[k], s->md, s->g, prescribed, s->d_err, s->stream);
    cudaEventRecord(s->bev[k], s->stream);  // this run's stage 1 and everything before it
    cudaStreamWaitEvent(s->stream2, s->bev[k], 0);
    launched += ms::launch_mol_stage2(runs[k], s->md, s->g, prescribed, s->d_err, s->stream2);
  }
  cudaEventRecord(s->bev[nrun], s->stream2);
  cudaStreamWaitEvent(s->stream, s->bev[nrun], 0);
  return launched;
}

static void step_once(ms_sim* s, float2* const* scratch, const FieldRecorder* rec = nullptr) {
  const bool fdtd = s->drive == MS_DRIVE_FDTD;
  // sub-stepping: the molecules advance (by nsub dt) on every nsub-th step only,
  // and only those steps' E updates take the molecular dipole change
  const bool molecular = s->steps % s->nsub == 0;
  int launched = 0;
  if (s->timing) mark(s);
  if (fdtd) {
    ms::launch_yee_h(s->g, s->stream);  // with the incident lines' H half step
    ++launched;
  }
  if (rec) {
    ms::launch_record_fields(s->g, s->md.cell, rec->ids, rec->m, rec->out, s->stream);
    ++launched;
  }
  if (s->timing) mark(s);
  ms::SpeciesDev sp[ms::kMaxSpecies];
  for (int si = 0; si < s->nspecies; ++si) {
    sp[si] = s->sp[si];
    if (scratch && sp[si].path == MS_MOL_STREAMING) sp[si].d2 = scratch[si];  // rewritten before it is read
  }
  if (molecular && s->batches > 0) {
    launched += pipelined_molecules(s, sp, fdtd ? 0 : 1);
    if (s->timing) mark(s);  // stages overlap: only the molecular phase as a whole is timed
  } else {
    if (molecular)
      for (int si = 0; si < s->nspecies; ++si)
        launched += ms::launch_mol_stage1(sp[si], s->md, s->g, fdtd ? 0 : 1, s->d_err, s->stream);
    if (s->timing) mark(s);
    if (molecular)
      for (int si = 0; si < s->nspecies; ++si)
        launched += ms::launch_mol_stage2(sp[si], s->md, s->g, fdtd ? 0 : 1, s->d_err, s->stream);
  }
  if (s->timing) mark(s);
  if (fdtd) {
    ms::Grid ge = s->g;
    if (!molecular) ge.mk1 = ge.mk0;  // no molecular slab: the dipoles did not change
    ms::launch_yee_e(ge, s->stream);  // with the incident lines' E half step
    ++launched;
    if (s->g.ndet > 0) {
      ms::launch_dft(s->g, s->stream);
      ++launched;
    }
  }
  if (s->timing) mark(s);  // the phases end here; the counter runs between steps
  ms::launch_step_counter(s->d_step, s->stream);
  ++launched;
  ++s->steps;
  if (s->timing) {
    s->timed_steps++;
    s->launches += launched;
  }
}

// Capture the launches of s->gsteps steps from phase 0 into a graph.  The
// host step count is restored: capturing runs nothing.
static ms_status capture_cycle(ms_sim* s) {
  if (s->gexec) cudaGraphExecDestroy(s->gexec);
  s->gexec = nullptr;
  s->gsteps = s->nsub * std::max(1, (8 + s->nsub - 1) / s->nsub);
  const int64_t saved = s->steps;
  if (cudaStreamBeginCapture(s->stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return MS_ECUDA;
  for (int q = 0; q < s->gsteps; ++q) step_once(s, nullptr);
  s->steps = saved;
  cudaGraph_t g = nullptr;
  const cudaError_t e = cudaStreamEndCapture(s->stream, &g);
  if (e != cudaSuccess || !g) {
    cudaGetLastError();
    return MS_ECUDA;
  }
  const cudaError_t ie = cudaGraphInstantiate(&s->gexec, g, 0);
  cudaGraphDestroy(g);
  if (ie != cudaSuccess) {
    cudaGetLastError();
    s->gexec = nullptr;
    return MS_ECUDA;
  }
  s->gdirty = false;
  return MS_OK;
}

ms_status ms_step(ms_sim* s, int64_t n) {
  if (!s || n < 0) return MS_EINVAL;
  if (s->drive == MS_DRIVE_PRESCRIBED && s->nmol > 0 && s->steps + n > s->nwave) return MS_EINVAL;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(s->stream, &cs) != cudaSuccess) return MS_ECUDA;
  if (s->graphs && !s->timing && cs == cudaStreamCaptureStatusNone) {
    while (n > 0 && s->steps % s->nsub != 0) {  // to the start of a molecular cycle
      step_once(s, nullptr);
      --n;
    }
    const int L = s->nsub * std::max(1, (8 + s->nsub - 1) / s->nsub);
    if (n >= L) {
      if (!s->gexec || s->gdirty || s->gsteps != L) MS_TRY(capture_cycle(s));
      for (; n >= L; n -= L) {
        if (cudaGraphLaunch(s->gexec, s->stream) != cudaSuccess) return MS_ECUDA;
        s->steps += L;
      }
    }
  }
  for (int64_t q = 0; q < n; ++q) step_once(s, nullptr);
  return cudaGetLastError() == cudaSuccess ? MS_OK : MS_ECUDA;
}

ms_status ms_step_noalloc(ms_sim* s, int64_t n) {
  if (!s || n < 0) return MS_EINVAL;
  if (s->drive == MS_DRIVE_PRESCRIBED && s->nmol > 0 && s->steps + n > s->nwave) return MS_EINVAL;
  // each streaming species gets its own region of the fixed array, at
  // 256-byte aligned offsets; all of them must fit (checked before any launch)
  float2* scratch[ms::kMaxSpecies] = {};
  size_t off = 0;
  for (int si = 0; si < s->nspecies; ++si) {
    const ms::SpeciesDev& sp = s->sp[si];
    if (sp.path != MS_MOL_STREAMING || sp.bloch || sp.nmol == 0) continue;
    const size_t bytes = (size_t)sp.nmol * sp.rows * sp.nr * sizeof(float2);
    if (bytes > kNoAllocScratchBytes || off > kNoAllocScratchBytes - bytes) return MS_EINVAL;
    scratch[si] = s->noalloc_base + off / sizeof(float2);
    off += (bytes + 255) / 256 * 256;
  }
  if (!s->noalloc_base) return MS_ECUDA;
  for (int64_t q = 0; q < n; ++q) step_once(s, scratch);
  return cudaGetLastError() == cudaSuccess ? MS_OK : MS_ECUDA;
}

ms_status ms_timing_begin(ms_sim* s) {
  if (!s) return MS_EINVAL;
  for (cudaEvent_t e : s->events) cudaEventDestroy(e);
  s->events.clear();
  s->timed_steps = 0;
  s->launches = 0;
  s->timing = true;
  return MS_OK;
}

ms_status ms_timing_end(ms_sim* s, double out[6], int64_t* steps, int64_t* launches) {
  if (!s || !out) return MS_EINVAL;
  s->timing = false;
  if (cudaStreamSynchronize(s->stream) != cudaSuccess) return MS_ECUDA;
  double acc[4] = {0, 0, 0, 0};  // H, stage 1, stage 2, E
  for (size_t b = 0; b + 4 < s->events.size(); b += 5)
    for (int p = 0; p < 4; ++p) {
      float ms = 0.f;
      if (cudaEventElapsedTime(&ms, s->events[b + p], s->events[b + p + 1]) != cudaSuccess) return MS_ECUDA;
      acc[p] += ms;
    }
  out[0] = acc[0];
  out[1] = acc[1] + acc[2];
  out[2] = acc[3];
  out[3] = acc[0] + acc[1] + acc[2] + acc[3];
  out[4] = acc[1];
  out[5] = acc[2];
  if (steps) *steps = s->timed_steps;
  if (launches) *launches = s->launches;
  for (cudaEvent_t e : s->events) cudaEventDestroy(e);
  s->events.clear();
  return MS_OK;
}

int64_t ms_step_count(const ms_sim* s) { return s ? s->steps : -1; }

ms_status ms_read_fields(ms_sim* s, int32_t which, int32_t sim, float* dst, size_t n) {
  if (!s || !dst || s->drive != MS_DRIVE_FDTD || sim < 0 || sim >= s->g.nsim) return MS_EINVAL;
  const size_t per = (size_t)s->g.ncell_sim;
  if (n < 3 * per || (which != MS_FIELD_E && which != MS_FIELD_H)) return MS_EINVAL;
  float* const* src = which == MS_FIELD_E ? s->g.E : s->g.H;
  for (int c = 0; c < 3; ++c)
    if (cudaMemcpyAsync(dst + c * per, src[c] + (size_t)sim * per, per * sizeof(float),
                        cudaMemcpyDeviceToHost, s->stream) != cudaSuccess)
      return MS_ECUDA;
  return latched(s);
}

ms_status ms_write_fields(ms_sim* s, int32_t which, int32_t sim, const float* src, size_t n) {
  if (!s || !src || s->drive != MS_DRIVE_FDTD || sim < 0 || sim >= s->g.nsim) return MS_EINVAL;
  const size_t per = (size_t)s->g.ncell_sim;
  if (n < 3 * per || (which != MS_FIELD_E && which != MS_FIELD_H)) return MS_EINVAL;
  float* const* dst = which == MS_FIELD_E ? s->g.E : s->g.H;
  for (int c = 0; c < 3; ++c)
    if (cudaMemcpyAsync(dst[c] + (size_t)sim * per, src + c * per, per * sizeof(float),
                        cudaMemcpyHostToDevice, s->stream) != cudaSuccess)
      return MS_ECUDA;
  return cudaStreamSynchronize(s->stream) == cudaSuccess ? MS_OK : MS_ECUDA;
}

static ms_status read_range(ms_sim* s, const double* dev, int width, int64_t first, int64_t count, double* dst) {
  if (!dst) return MS_OK;
  if (cudaMemcpyAsync(dst, dev + (size_t)width * first, (size_t)width * count * sizeof(double),
                      cudaMemcpyDeviceToHost, s->stream) != cudaSuccess)
    return MS_ECUDA;
  return MS_OK;
}

static ms_status read_pairs(ms_sim* s, const double* dev, int64_t first, int64_t count, double* a, double* b) {
  if (!a && !b) return MS_OK;
  std::vector<double> tmp(2 * (size_t)count);
  MS_TRY(read_range(s, dev, 2, first, count, tmp.data()));
  if (cudaStreamSynchronize(s->stream) != cudaSuccess) return MS_ECUDA;
  for (int64_t q = 0; q < count; ++q) {
    if (a) a[q] = tmp[2 * q];
    if (b) b[q] = tmp[2 * q + 1];
  }
  return MS_OK;
}

ms_status ms_read_populations(ms_sim* s, int64_t first, int64_t count, double* Pg, double* Pe) {
  if (!s || first < 0 || count < 0 || first + count > s->nmol) return MS_EINVAL;
  MS_TRY(read_pairs(s, s->md.pop, first, count, Pg, Pe));
  return latched(s);
}

ms_status ms_read_dissociation(ms_sim* s, int64_t first, int64_t count, double* ag, double* ae,
                               double* Rnum, double* Rden) {
  if (!s || first < 0 || count < 0 || first + count > s->nmol) return MS_EINVAL;
  MS_TRY(read_pairs(s, s->md.absorbed, first, count, ag, ae));
  if (Rnum || Rden) {
    for (int si = 0; si < s->nspecies; ++si) ms::launch_mol_observe(s->sp[si], s->md, s->stream);
    if (cudaGetLastError() != cudaSuccess) return MS_ECUDA;
    MS_TRY(read_range(s, s->md.Rnum, 1, first, count, Rnum));
    MS_TRY(read_range(s, s->md.Rden, 1, first, count, Rden));
  }
  return latched(s);
}

ms_status ms_read_dipoles(ms_sim* s, int64_t first, int64_t count, double* mu) {
  if (!s || !mu || first < 0 || count < 0 || first + count > s->nmol) return MS_EINVAL;
  MS_TRY(read_range(s, s->md.mu, 3, first, count, mu));
  return latched(s);
}

ms_status ms_set_prescribed_field(ms_sim* s, const float* amp, const float* wave, int64_t nsteps) {
  if (!s || !amp || !wave || nsteps <= 0 || s->drive != MS_DRIVE_PRESCRIBED) return MS_EINVAL;
  s->gdirty = true;
  if (s->md.amp == nullptr) MS_TRY(upload(s, (float**)&s->md.amp, amp, 3 * (size_t)(s->nmol > 0 ? s->nmol : 1)));
  else if (cudaMemcpyAsync((void*)s->md.amp, amp, 3 * sizeof(float) * s->nmol, cudaMemcpyHostToDevice, s->stream) != cudaSuccess)
    return MS_ECUDA;
  float* w = nullptr;
  MS_TRY(upload(s, &w, wave, (size_t)nsteps));
  s->md.wave = w;
  s->md.nwave = nsteps;
  s->nwave = nsteps;
  return cudaStreamSynchronize(s->stream) == cudaSuccess ? MS_OK : MS_ECUDA;
}

ms_status ms_set_replay_field(ms_sim* s, const float* E, int64_t nsteps) {
  if (!s || !E || nsteps <= 0 || s->drive != MS_DRIVE_PRESCRIBED) return MS_EINVAL;
  s->gdirty = true;
  float* d = nullptr;
  MS_TRY(upload(s, &d, E, (size_t)nsteps * 3 * (size_t)(s->nmol > 0 ? s->nmol : 1)));
  s->md.replay = d;
  s->md.nwave = nsteps;
  s->nwave = nsteps;
  return cudaStreamSynchronize(s->stream) == cudaSuccess ? MS_OK : MS_ECUDA;
}

ms_status ms_record_local_fields(ms_sim* s, const int64_t* mol_ids, int64_t m, float* dst, int64_t nsteps) {
  if (!s || !mol_ids || !dst || m <= 0 || m > INT32_MAX || nsteps < 0 || s->drive != MS_DRIVE_FDTD) return MS_EINVAL;
  for (int64_t k = 0; k < m; ++k)
    if (mol_ids[k] < 0 || mol_ids[k] >= s->nmol) return MS_EINVAL;
  if (nsteps == 0) return latched(s);
  // temporary device buffers: ids and [nsteps][m][3] samples, released before returning
  const size_t nid = (size_t)m * sizeof(long long), nout = (size_t)nsteps * m * 3 * sizeof(float);
  void *d_ids = nullptr, *d_out = nullptr;
  auto tmp_free = [&](void* p) {
    if (!p) return;
    if (s->al.fr) s->al.fr(p, s->al.ctx);
    else cudaFree(p);
  };
  auto tmp_alloc = [&](size_t n) -> void* {
    void* p = nullptr;
    if (s->al.fn) p = s->al.fn(n, s->al.ctx);
    else if (cudaMalloc(&p, n) != cudaSuccess) {
      cudaGetLastError();
      p = nullptr;
    }
    return p;
  };
  d_ids = tmp_alloc(nid);
  d_out = tmp_alloc(nout);
  ms_status st = MS_OK;
  if (!d_ids || !d_out) st = MS_ENOMEM;
  std::vector<long long> ids(mol_ids, mol_ids + m);
  if (st == MS_OK && cudaMemcpyAsync(d_ids, ids.data(), nid, cudaMemcpyHostToDevice, s->stream) != cudaSuccess)
    st = MS_ECUDA;
  if (st == MS_OK) {
    FieldRecorder rec{static_cast<const long long*>(d_ids), (int)m, static_cast<float*>(d_out)};
    for (int64_t q = 0; q < nsteps; ++q) {
      step_once(s, nullptr, &rec);
      rec.out += (size_t)m * 3;
    }
    if (cudaGetLastError() != cudaSuccess ||
        cudaMemcpyAsync(dst, d_out, nout, cudaMemcpyDeviceToHost, s->stream) != cudaSuccess ||
        cudaStreamSynchronize(s->stream) != cudaSuccess)
      st = MS_ECUDA;
  }
  cudaStreamSynchronize(s->stream);
  tmp_free(d_ids);
  tmp_free(d_out);
  return st == MS_OK ? latched(s) : st;
}

// ---- spectral detection ----------------------------------------------------
ms_status ms_set_detectors(ms_sim* s, const int32_t* planes_z, int32_t nplanes, const double* omega,
                           int32_t nfreq) {
  if (!s || !planes_z || !omega || s->drive != MS_DRIVE_FDTD || nplanes < 1 || nplanes > 16 || nfreq < 1 ||
      nfreq > 512)
    return MS_EINVAL;
  s->gdirty = true;
  for (int d = 0; d < nplanes; ++d)
    if (planes_z[d] < 1 || planes_z[d] >= s->g.nz - 1) return MS_EINVAL;
  for (int f = 0; f < nfreq; ++f)
    if (!std::isfinite(omega[f])) return MS_EINVAL;
  if (cudaStreamSynchronize(s->stream) != cudaSuccess) return MS_ECUDA;
  int* dk = nullptr;
  double* dw = nullptr;
  double2* acc = nullptr;
  std::vector<int> k(planes_z, planes_z + nplanes);
  std::vector<double> w(omega, omega + nfreq);
  MS_TRY(upload(s, &dk, k.data(), k.size()));
  MS_TRY(upload(s, &dw, w.data(), w.size()));
  MS_TRY(zeros(s, &acc, (size_t)s->g.nsim * nplanes * nfreq * 4 * s->g.nx * s->g.ny));
  s->g.det_k = dk;
  s->g.omega = dw;
  s->g.dft = acc;
  s->g.ndet = nplanes;
  s->g.nfreq = nfreq;
  return cudaStreamSynchronize(s->stream) == cudaSuccess ? MS_OK : MS_ECUDA;
}

ms_status ms_read_dft(ms_sim* s, int32_t plane, int32_t sim_index, int32_t component, int32_t freq,
                      double* dst) {
  if (!s || !dst || plane < 0 || plane >= s->g.ndet || sim_index < 0 || sim_index >= s->g.nsim ||
      component < 0 || component > 3 || freq < 0 || freq >= s->g.nfreq)
    return MS_EINVAL;
  const size_t cells = (size_t)s->g.nx * s->g.ny;
  const double2* src =
      s->g.dft + ((((size_t)sim_index * s->g.ndet + plane) * s->g.nfreq + freq) * 4 + component) * cells;
  if (cudaMemcpyAsync(dst, src, cells * sizeof(double2), cudaMemcpyDeviceToHost, s->stream) != cudaSuccess)
    return MS_ECUDA;
  return latched(s);
}

ms_status ms_read_flux(ms_sim* s, int32_t plane, double* flux) {
  if (!s || !flux || plane < 0 || plane >= s->g.ndet) return MS_EINVAL;
  const size_t cells = (size_t)s->g.nx * s->g.ny, nf = (size_t)s->g.nfreq;
  std::vector<double2> a(4 * cells);
  const double dx2 = s->dx * s->dx;
  for (int sim = 0; sim < s->g.nsim; ++sim)
    for (size_t f = 0; f < nf; ++f) {
      const double2* src = s->g.dft + ((((size_t)sim * s->g.ndet + plane) * nf + f) * 4) * cells;
      if (cudaMemcpyAsync(a.data(), src, 4 * cells * sizeof(double2), cudaMemcpyDeviceToHost, s->stream) !=
              cudaSuccess ||
          cudaStreamSynchronize(s->stream) != cudaSuccess)
        return MS_ECUDA;
      double acc = 0.0;  // Re (Ex conj(Hy) - Ey conj(Hx))
      for (size_t q = 0; q < cells; ++q) {
        const double2 ex = a[q], ey = a[cells + q], hx = a[2 * cells + q], hy = a[3 * cells + q];
        acc += (ex.x * hy.x + ex.y * hy.y) - (ey.x * hx.x + ey.y * hx.y);
      }
      flux[(size_t)sim * nf + f] = acc * dx2;
    }
  return latched(s);
}

// ---- checkpoint ------------------------------------------------------------
namespace {
constexpr char kCkMagic[8] = {'M', 'S', '2', '2', '0', '9', 'C', 'K'};
constexpr uint32_t kCkVersion = 4;

struct CkHeader {
  char magic[8];
  uint32_t version, drive;
  int64_t steps;
  int32_t nx, ny, nz, nsim;
  int64_t nmol;
  int32_t nspecies, pml, ks, jk0, jk1, aux_len;
  int32_t ndet, nfreq, state_rows[ms::kMaxSpecies];
  int32_t mol_substeps, src_kind;
  int32_t species[ms::kMaxSpecies][3];  // nr, jmax, molecules
  uint64_t nblobs;
};

struct Blob {
  void* ptr;
  size_t bytes;
};

// The evolving device state of a handle, in a fixed order.
std::vector<Blob> state_blobs(ms_sim* s) {
  std::vector<Blob> b;
  const ms::Grid& g = s->g;
  if (s->drive == MS_DRIVE_FDTD) {
    const size_t ncell = (size_t)g.ncell_sim * g.nsim;
    for (int c = 0; c < 3; ++c) b.push_back({g.E[c], ncell * sizeof(float)});
    for (int c = 0; c < 3; ++c) b.push_back({g.H[c], ncell * sizeof(float)});
    const size_t nj = (size_t)g.nsim * (g.jk1 - g.jk0) * g.nx * g.ny;
    if (nj > 0)
      for (int c = 0; c < 3; ++c) b.push_back({g.J[c], nj * sizeof(float)});
    if (g.pml > 0) {
      const size_t np = (size_t)g.nsim * 2 * g.pml * g.nx * g.ny;
      for (int c = 0; c < 2; ++c) b.push_back({g.psiE[c], np * sizeof(float)});
      for (int c = 0; c < 2; ++c) b.push_back({g.psiH[c], np * sizeof(float)});
    }
    if (g.ks >= 0) {
      b.push_back({g.auxE, (size_t)g.nsim * (g.aux_len + 1) * sizeof(float)});
      b.push_back({g.auxH, (size_t)g.nsim * g.aux_len * sizeof(float)});
    }
    if (g.ndet > 0)
      b.push_back({g.dft, (size_t)g.nsim * g.ndet * g.nfreq * 4 * g.nx * g.ny * sizeof(double2)});
  }
  for (int si = 0; si < s->nspecies; ++si) {
    const ms::SpeciesDev& sp = s->sp[si];
    if (sp.bloch) b.push_back({sp.bloch_y, (size_t)sp.nmol * 3 * sizeof(double)});
    else b.push_back({sp.psi, (size_t)sp.nmol * sp.rows * sp.nr * sizeof(float2)});
  }
  if (s->nmol > 0) {
    const size_t n = (size_t)s->nmol;
    b.push_back({s->md.mu, 3 * n * sizeof(double)});
    b.push_back({s->md.dmu, 3 * n * sizeof(double)});
    b.push_back({s->md.pop, 2 * n * sizeof(double)});
    b.push_back({s->md.absorbed, 2 * n * sizeof(double)});
    b.push_back({s->md.ncorr, n * sizeof(float)});
  }
  return b;
}

CkHeader make_header(ms_sim* s, uint64_t nblobs) {
  CkHeader h;
  std::memset(&h, 0, sizeof(h));
  std::memcpy(h.magic, kCkMagic, 8);
  h.version = kCkVersion;
  h.drive = (uint32_t)s->drive;
  h.steps = s->steps;
  h.nx = s->g.nx;
  h.ny = s->g.ny;
  h.nz = s->g.nz;
  h.nsim = s->g.nsim;
  h.nmol = s->nmol;
  h.nspecies = s->nspecies;
  h.pml = s->g.pml;
  h.ks = s->g.ks;
  h.jk0 = s->g.jk0;
  h.jk1 = s->g.jk1;
  h.aux_len = s->g.aux_len;
  h.ndet = s->g.ndet;
  h.nfreq = s->g.nfreq;
  for (int si = 0; si < s->nspecies; ++si) h.state_rows[si] = s->sp[si].rows;
  h.mol_substeps = s->nsub;
  h.src_kind = s->src_kind;
  for (int si = 0; si < s->nspecies; ++si) {
    h.species[si][0] = s->sp[si].nr;
    h.species[si][1] = s->sp[si].jmax;
    h.species[si][2] = s->sp[si].nmol;
  }
  h.nblobs = nblobs;
  return h;
}

constexpr size_t kCkChunk = 64u << 20;  // host staging buffer

// Two pinned staging buffers for checkpoint I/O: the copy between the device
// and one buffer overlaps the file transfer of the other.  ok = false (the
// pageable path is used) when pinned memory cannot be had.
struct PinnedPair {
  char* p[2] = {nullptr, nullptr};
  cudaEvent_t ev[2] = {nullptr, nullptr};
  bool ok = false;
  PinnedPair() {
    ok = true;
    for (int i = 0; i < 2 && ok; ++i)
      ok = cudaHostAlloc(reinterpret_cast<void**>(&p[i]), kCkChunk, cudaHostAllocDefault) == cudaSuccess &&
           cudaEventCreateWithFlags(&ev[i], cudaEventDisableTiming) == cudaSuccess;
    if (!ok) cudaGetLastError();
  }
  ~PinnedPair() {
    for (int i = 0; i < 2; ++i) {
      if (ev[i]) {
        cudaEventSynchronize(ev[i]);  // no copy still reads or writes the buffer
        cudaEventDestroy(ev[i]);
      }
      if (p[i]) cudaFreeHost(p[i]);
    }
  }
};
}  // namespace

ms_status ms_save(ms_sim* s, const char* path) {
  if (!s || !path) return MS_EINVAL;
  if (cudaStreamSynchronize(s->stream) != cudaSuccess) return MS_ECUDA;
  const std::vector<Blob> blobs = state_blobs(s);
  const CkHeader h = make_header(s, blobs.size());
  FILE* f = std::fopen(path, "wb");
  if (!f) return MS_EIO;
  ms_status st = std::fwrite(&h, sizeof(h), 1, f) == 1 ? MS_OK : MS_EIO;
  PinnedPair pin;
  std::vector<char> buf;
  for (size_t k = 0; st == MS_OK && k < blobs.size(); ++k) {
    const uint64_t nb = blobs[k].bytes;
    if (std::fwrite(&nb, sizeof(nb), 1, f) != 1) {
      st = MS_EIO;
      break;
    }
    if (pin.ok) {  // chunk c copies into buffer c & 1 while chunk c - 1 is written out
      size_t prev_len = 0;
      int c = 0;
      for (size_t off = 0; st == MS_OK && off < nb; off += kCkChunk, ++c) {
        const size_t len = std::min(kCkChunk, (size_t)nb - off);
        const int b = c & 1;
        if (cudaEventSynchronize(pin.ev[b]) != cudaSuccess ||
            cudaMemcpyAsync(pin.p[b], static_cast<char*>(blobs[k].ptr) + off, len, cudaMemcpyDeviceToHost,
                            s->stream) != cudaSuccess ||
            cudaEventRecord(pin.ev[b], s->stream) != cudaSuccess) {
          st = MS_ECUDA;
          break;
        }
        if (c > 0) {
          if (cudaEventSynchronize(pin.ev[b ^ 1]) != cudaSuccess) st = MS_ECUDA;
          else if (std::fwrite(pin.p[b ^ 1], 1, prev_len, f) != prev_len) st = MS_EIO;
        }
        prev_len = len;
      }
      if (st == MS_OK && c > 0) {
        const int b = (c - 1) & 1;
        if (cudaEventSynchronize(pin.ev[b]) != cudaSuccess) st = MS_ECUDA;
        else if (std::fwrite(pin.p[b], 1, prev_len, f) != prev_len) st = MS_EIO;
      }
      continue;
    }
    for (size_t off = 0; off < nb; off += kCkChunk) {
      const size_t len = std::min(kCkChunk, (size_t)nb - off);
      buf.resize(len);
      if (cudaMemcpy(buf.data(), static_cast<char*>(blobs[k].ptr) + off, len, cudaMemcpyDeviceToHost) !=
          cudaSuccess) {
        st = MS_ECUDA;
        break;
      }
      if (std::fwrite(buf.data(), 1, len, f) != len) {
        st = MS_EIO;
        break;
      }
    }
  }
  if (std::fclose(f) != 0 && st == MS_OK) st = MS_EIO;
  return st == MS_OK ? latched(s) : st;
}

ms_status ms_load(ms_sim* s, const char* path) {
  if (!s || !path) return MS_EINVAL;
  if (cudaStreamSynchronize(s->stream) != cudaSuccess) return MS_ECUDA;
  const std::vector<Blob> blobs = state_blobs(s);
  const CkHeader want = make_header(s, blobs.size());
  FILE* f = std::fopen(path, "rb");
  if (!f) return MS_EIO;
  CkHeader h;
  ms_status st = MS_OK;
  if (std::fread(&h, sizeof(h), 1, f) != 1 || std::memcmp(h.magic, kCkMagic, 8) != 0 || h.version != kCkVersion)
    st = MS_EIO;
  else {
    CkHeader a = h, b = want;  // compare everything but the step count
    a.steps = b.steps = 0;
    if (std::memcmp(&a, &b, sizeof(a)) != 0) st = MS_EINVAL;
  }
  PinnedPair pin;
  std::vector<char> buf;
  for (size_t k = 0; st == MS_OK && k < blobs.size(); ++k) {
    uint64_t nb = 0;
    if (std::fread(&nb, sizeof(nb), 1, f) != 1) {
      st = MS_EIO;
      break;
    }
    if (nb != blobs[k].bytes) {
      st = MS_EINVAL;
      break;
    }
    if (pin.ok) {  // chunk c is read into buffer c & 1 while chunk c - 1 copies to the device
      int c = 0;
      for (size_t off = 0; off < nb; off += kCkChunk, ++c) {
        const size_t len = std::min(kCkChunk, (size_t)nb - off);
        const int b = c & 1;
        if (cudaEventSynchronize(pin.ev[b]) != cudaSuccess) {
          st = MS_ECUDA;
          break;
        }
        if (std::fread(pin.p[b], 1, len, f) != len) {
          st = MS_EIO;
          break;
        }
        if (cudaMemcpyAsync(static_cast<char*>(blobs[k].ptr) + off, pin.p[b], len, cudaMemcpyHostToDevice,
                            s->stream) != cudaSuccess ||
            cudaEventRecord(pin.ev[b], s->stream) != cudaSuccess) {
          st = MS_ECUDA;
          break;
        }
      }
      continue;
    }
    for (size_t off = 0; off < nb; off += kCkChunk) {
      const size_t len = std::min(kCkChunk, (size_t)nb - off);
      buf.resize(len);
      if (std::fread(buf.data(), 1, len, f) != len) {
        st = MS_EIO;
        break;
      }
      if (cudaMemcpy(static_cast<char*>(blobs[k].ptr) + off, buf.data(), len, cudaMemcpyHostToDevice) !=
          cudaSuccess) {
        st = MS_ECUDA;
        break;
      }
    }
  }
  std::fclose(f);
  if (cudaStreamSynchronize(s->stream) != cudaSuccess && st == MS_OK) st = MS_ECUDA;  // copies in flight
  if (st != MS_OK) return st;
  // the step counter, host and device
  const long long step = h.steps;
  if (cudaMemcpy(s->g.step, &step, sizeof(step), cudaMemcpyHostToDevice) != cudaSuccess) return MS_ECUDA;
  s->steps = h.steps;
  return latched(s);
}

ms_status ms_check_bounded_wait(int32_t tries) {
  if (tries < 1 || tries > 100000) return MS_EINVAL;
  int* d_flag = nullptr;
  if (cudaMalloc(&d_flag, sizeof(int)) != cudaSuccess) {
    cudaGetLastError();
    return MS_ENOMEM;
  }
  int flag = 0;
  ms_status st = MS_OK;
  if (cudaMemset(d_flag, 0, sizeof(int)) != cudaSuccess || ms::launch_wait_timeout_probe(tries, d_flag, 0) != cudaSuccess ||
      cudaMemcpy(&flag, d_flag, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
    st = MS_ECUDA;
  cudaFree(d_flag);
  if (st != MS_OK) return st;
  return (flag & ms::kErrTimeout) ? MS_ETIMEOUT : MS_OK;
}

int32_t ms_species_path(const ms_sim* s, int32_t species) {
  if (!s || species < 0 || species >= s->nspecies) return MS_EINVAL;
  return s->sp[species].path;
}

ms_status ms_species_plan(const ms_sim* s, int32_t species, int32_t* path, int32_t* kernel, int32_t* chunk) {
  if (!s || !path || !kernel || !chunk || species < 0 || species >= s->nspecies) return MS_EINVAL;
  const ms::SpeciesDev& sp = s->sp[species];
  *path = sp.path;
  *kernel = sp.kern;
  *chunk = sp.ch;
  return MS_OK;
}

ms_status ms_species_plan_ex(const ms_sim* s, int32_t species, int32_t plan[4]) {
  if (!plan) return MS_EINVAL;
  MS_TRY(ms_species_plan(s, species, &plan[0], &plan[1], &plan[2]));
  plan[3] = s->sp[species].cps;
  return MS_OK;
}

ms_status ms_set_species_plan_ex(ms_sim* s, int32_t species, const int32_t plan[4]) {
  if (!s || !plan || species < 0 || species >= s->nspecies) return MS_EINVAL;
  const int32_t path = plan[0], kernel = plan[1], chunk = plan[2], cps = plan[3];
  ms::SpeciesDev& sp = s->sp[species];
  if (sp.bloch) return MS_EINVAL;
  const bool tiled = kernel == MS_KERN_TILE || kernel == MS_KERN_PAIR;
  if (cps < -1 || cps > 32 || (cps != 0 && !tiled)) return MS_EINVAL;
  int cand[32][4];
  const int nc = ms::mol_plan_candidates(sp, cand, 32);
  bool ok = false;
  if (kernel == MS_KERN_DEFAULT && chunk == 0) {
    for (int c = 0; c < nc; ++c) ok = ok || cand[c][0] == path;
    ok = ok || path == sp.path;  // the layout it already runs
  } else {
    for (int c = 0; c < nc; ++c)  // a tiled plan with chunk 0 follows the kernel's tile-width rule
      ok = ok || (cand[c][0] == path && cand[c][1] == kernel &&
                  (cand[c][2] == chunk || (tiled && chunk == 0)));
  }
  if (!ok) return MS_EINVAL;
  if (cudaStreamSynchronize(s->stream) != cudaSuccess) return MS_ECUDA;
  ms::SpeciesDev trial = sp;
  trial.path = path;
  if (path == MS_MOL_STREAMING) MS_TRY(ensure_scratch(s, trial));
  sp = trial;
  sp.kern = kernel;
  sp.ch = chunk;
  sp.cps = cps;
  s->gdirty = true;
  return MS_OK;
}

ms_status ms_set_species_plan(ms_sim* s, int32_t species, int32_t path, int32_t kernel, int32_t chunk) {
  const int32_t plan[4] = {path, kernel, chunk, 0};
  return ms_set_species_plan_ex(s, species, plan);
}

ms_status ms_set_mol_batches(ms_sim* s, int32_t batches) {
  if (!s || batches < 0 || batches > kMaxMolBatches) return MS_EINVAL;
  if (cudaStreamSynchronize(s->stream) != cudaSuccess) return MS_ECUDA;
  if (batches > 0) {  // the second stream and the event pool (completed by a later call if one failed)
    if (!s->stream2 && cudaStreamCreateWithFlags(&s->stream2, cudaStreamNonBlocking) != cudaSuccess) {
      cudaGetLastError();
      s->stream2 = nullptr;
      return MS_ECUDA;
    }
    const size_t nev = (size_t)ms::kMaxSpecies * kMaxMolBatches + 1;  // one per run, one for the join
    while (s->bev.size() < nev) {
      cudaEvent_t e = nullptr;
      if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) {
        cudaGetLastError();
        return MS_ECUDA;  // batches unchanged: the step stays sequential
      }
      s->bev.push_back(e);
    }
  }
  s->batches = batches;
  s->gdirty = true;
  return MS_OK;
}

int32_t ms_mol_batches(const ms_sim* s) { return s ? s->batches : -1; }

size_t ms_device_bytes(const ms_sim* s) { return s ? s->bytes : 0; }

void ms_destroy(ms_sim* s) {
  if (!s) return;
  s->release();
  delete s;
}

}  // extern "C"
