/*
 * ms.h -- C ABI of the GB300 coupled Maxwell-Schroedinger time step.
 *
 * The library advances, on one GPU, the coupled system of arXiv 2209.04487:
 *   - Maxwell's curl equations on a 3D Yee grid (Eq. 1), leap-frog, with a
 *     Drude current in metal cells (Eq. 2), periodic x/y, convolutional PML
 *     along z and a total-field/scattered-field plane-wave source
 *     (section "The domain decomposition methodology for FDTD");
 *   - an ensemble of diatomic molecules, each carrying ro-vibrational
 *     wavepackets xi^{g,e}_{jm}(R) on a ground and an excited surface
 *     (Eq. 3), advanced by split-operator steps of Eq. 4 with the effective
 *     Hamiltonians of Eq. 5 (Morse ground surface Eq. 6, repulsive excited
 *     surface of the Eq. 7 family, constant transition dipole or a given
 *     d(R)) under the local field E^n at the molecule's cell, every step or
 *     every N-th step by N dt; or frozen two-level molecules (Bloch
 *     equations, RK4; the scaling-experiments section);
 *   - the induced dipoles, multiplied by the molecular number density
 *     (one molecule per molecule: 1/dx^3 per cell), enter Ampere's law as
 *     the polarization current dP/dt (section "Efficient numerical
 *     implementation of quantum dynamics ...").
 *
 * Conventions (all calls):
 *   - Every input pointer is host memory owned by the caller; ms_create
 *     copies what it needs, so the caller may free its buffers afterwards.
 *   - Every output pointer is host memory allocated by the caller.
 *   - Calls return an ms_status and never throw or abort.  A device-side
 *     condition (non-finite field, coupling series that does not converge)
 *     is latched in a device word and reported by the next ms_step or
 *     ms_read_* call as MS_ENUMERIC.
 *   - ms_step is asynchronous on the handle's stream; ms_read_* synchronise
 *     that stream.  One handle must not be used from two threads at once.
 *   - There is no CPU fallback: without a compute-capability-10.3 device
 *     ms_create returns MS_EUNSUPPORTED.
 *
 * Array layouts:
 *   grid arrays are [nsim][nz][ny][nx] with x fastest; cell (i,j,k) owns
 *   Ex(i+1/2,j,k), Ey(i,j+1/2,k), Ez(i,j,k+1/2), Hx(i,j+1/2,k+1/2),
 *   Hy(i+1/2,j,k+1/2), Hz(i+1/2,j+1/2,k).  E is in V/m at integer steps,
 *   H in A/m at half steps.  Molecular quantities are in atomic units.
 */
#ifndef MS_H
#define MS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ms_sim ms_sim; /* opaque; owned by the library */

typedef enum {
  MS_OK = 0,
  MS_EINVAL = -1,       /* invalid descriptor or argument */
  MS_ENOMEM = -2,       /* device allocation failed (nothing leaked) */
  MS_ECUDA = -3,        /* a CUDA runtime call failed */
  MS_ENUMERIC = -4,     /* latched device condition: non-finite value or
                           a coupling exponential that did not converge */
  MS_ETIMEOUT = -5,     /* a bounded device wait on an asynchronous copy gave up */
  MS_EUNSUPPORTED = -6, /* no sm_103 device, or a configuration this build
                           does not support */
  MS_EIO = -7           /* a checkpoint file could not be written or read,
                           or is not a checkpoint of this library */
} ms_status;

enum { MS_BC_PML = 0, MS_BC_PERIODIC = 1 };
/* Arithmetic of the kinetic pass (the section on the split-operator
 * propagator).  MS_PREC_FP32: FP32 FFTs.  MS_PREC_MIXED_F16X3: the circulant
 * (K - I) applied to every state row as a tensor-core GEMM on split FP16
 * operands (x = hi + lo after an exact power-of-two scaling of each row and
 * of the matrix, three products hi*hi + hi*lo + lo*hi, FP32 accumulation),
 * which carries about 22 bits of each operand; the streaming layout only,
 * N_r 64 or 128 (MS_EUNSUPPORTED otherwise). */
enum { MS_PREC_FP32 = 0, MS_PREC_MIXED_F16X3 = 1 };
enum { MS_DRIVE_FDTD = 0, MS_DRIVE_PRESCRIBED = 1 };
enum { MS_FIELD_E = 0, MS_FIELD_H = 1 };
/* Molecular kernel layout.  MS_MOL_FUSED keeps each molecule's state in
 * shared memory for the whole step, so the state is read and written once
 * per step (species whose state fits, up to J = 8 at N_r = 64).
 * MS_MOL_STREAMING runs the kinetic pass over blocks of rows into a device
 * scratch buffer of the state's size, then streams state and scratch
 * through the R-space pass (any species up to J = 16, and the mixed
 * precision form).  MS_MOL_AUTO picks the fused form for FP32 species with
 * J <= 4 at N_r = 128 (its point-resident kernel), else the streaming
 * form. */
enum { MS_MOL_AUTO = 0, MS_MOL_FUSED = 1, MS_MOL_STREAMING = 2 };
/* Stored rows of each molecule's state.  MS_STATE_FULL: both surfaces carry
 * every channel (j, m), j <= J.  MS_STATE_PARITY: only (ground, even j) and
 * (excited, odd j), the only rows the dynamics populate from the j = 0
 * ground-state start (each coupling changes j by one and swaps the
 * surfaces), which halves the state and the work.  Results are those of the
 * full state.  Up to J = 4 the point-resident kernels run them (the fused
 * layout only at N_r = 128); from J = 5 on the two-points-a-thread tiled
 * kernel in the streaming layout with the FP32 kinetic pass (MS_EUNSUPPORTED
 * otherwise).  Their plan follows this rule (ms_set_species_plan accepts no
 * other). */
enum { MS_STATE_FULL = 0, MS_STATE_PARITY = 1 };
/* Step replay.  MS_GRAPHS_AUTO: ms_step captures the launches of whole
 * molecular cycles (at least 8 field steps, a multiple of mol_substeps) once
 * into a CUDA graph and replays it, and runs leftover steps eagerly; it runs
 * every step eagerly while phase timing is on or when the stream is already
 * being captured by the caller.  MS_GRAPHS_OFF: always eager.  Both give the
 * same results bit for bit. */
enum { MS_GRAPHS_AUTO = 0, MS_GRAPHS_OFF = 1 };
/* A species' plan: its layout (MS_MOL_FUSED or MS_MOL_STREAMING) and the
 * kernel of its R-space pass.  MS_KERN_POINT: one CTA of 2 N_r threads per
 * molecule, thread = (radial point, surface) (J <= 4; fused at N_r 128).
 * MS_KERN_TILE: persistent CTAs that each walk a share of the molecules, one
 * molecule at a time over tiles of `chunk` radial points of all rows, staged
 * by tensor copies (streaming; chunk 32 or 16 for J <= 8, 8 for J 9..16;
 * chunk 0: 8 from J = 9 on, 16 from J = 5 on, else 32).  MS_KERN_CHUNK: one CTA per molecule over chunks of `chunk`
 * radial points (4, 8, 16 or 32) of all rows (any J).  MS_KERN_PAIR: the
 * tiled kernel's schedule with two neighbouring radial points per thread and
 * packed FP32x2 arithmetic (streaming; chunk 32 or 16 for J <= 4, 16 or 8
 * for J 5..8, 8 for J 9..16; chunk 0: 8 from J = 5 on, else 32; the
 * parity-reduced state: 16 for J 5..8).  MS_KERN_DEFAULT: the
 * static rule (the first that applies of point for J <= 4, pair from J = 5
 * on in the streaming layout, tile, chunk at the widest fitting chunk).
 * Parity-reduced and d(R) species run
 * the point-resident kernel only.  Every plan computes the same step; their
 * results differ by FP32 rounding.
 * Autotuning (ms_options.autotune = MS_TUNE_MEASURE): ms_create times every
 * plan a species can run on a sandbox copy of up to 2,048 of its molecules
 * under a strong prescribed field (5e9 V/m, the coupling series' term count
 * of a pulse peak) and keeps the fastest; ms_species_plan reports the choice and
 * ms_set_species_plan pins one, so a tuned choice can be replayed. */
enum { MS_KERN_DEFAULT = 0, MS_KERN_POINT = 1, MS_KERN_TILE = 2, MS_KERN_CHUNK = 3, MS_KERN_PAIR = 4 };
enum { MS_TUNE_OFF = 0, MS_TUNE_MEASURE = 1 };

/* Grid and source.  dt must satisfy dt <= dx/(sqrt(3) c) (checked).
 * src_plane_z: absolute z index of the TF/SF plane (total field for
 * k >= src_plane_z), -1 for no source; it must lie outside the z absorbers.
 * The incident plane wave is x-polarised and travels towards +z; its value
 * at the plane, with w the carrier's angular frequency, is
 *   MS_SRC_PULSE (Sec. 3's femtosecond pulses): src rows (peak field E0
 *     [V/m], carrier photon energy [eV], FWHM of the field envelope [s],
 *     time of the peak t0 [s]);
 *     E(t) = E0 exp(-4 ln2 ((t-t0)/fwhm)^2) cos(w (t-t0));
 *   MS_SRC_CW (Sec. 3's continuous-wave drive): src rows (E0 [V/m], carrier
 *     photon energy [eV], turn-on time t_on [s], phase reference t0 [s]);
 *     E(t) = E0 sin^2(pi t / (2 t_on)) cos(w (t-t0)) for t < t_on, then
 *     E0 cos(w (t-t0)).
 * fwhm and t_on must be > 0 (MS_EINVAL otherwise). */
enum { MS_SRC_PULSE = 0, MS_SRC_CW = 1 };
typedef struct {
  int32_t nx, ny, nz, nsim;
  double dx_m, dt_s;
  int32_t pml_cells;   /* CPML thickness at each z end (MS_BC_PML) */
  int32_t bc_z;        /* MS_BC_PML or MS_BC_PERIODIC */
  int32_t src_plane_z; /* -1 = no source */
  const double* src;   /* [nsim][4], may be NULL when src_plane_z < 0 */
  int32_t src_kind;    /* MS_SRC_PULSE or MS_SRC_CW */
} ms_grid_desc;

/* Materials: n_materials entries of (eps_inf, plasma energy wp [eV],
 * damping gamma [eV]); wp = 0 marks a non-dispersive dielectric with
 * eps = eps_inf.  material_id: [nsim][nz][ny][nx] bytes, < n_materials. */
typedef struct {
  int32_t n_materials;
  const double* eps_inf;
  const double* wp_eV;
  const double* gamma_eV;
  const uint8_t* material_id;
} ms_materials_desc;

/* One molecular species (atomic units).
 *
 * MS_MODEL_WAVEPACKET (Eqs. 3-7): radial grid r_i = rmin + i dR,
 * dR = (rmax - rmin)/(nr - 1), nr in {64, 128, 256}; rotational channels
 * j <= jmax, |m| <= j ((jmax+1)^2 per surface), jmax <= 16.
 * Ground surface De (1 - exp(-a (r - re)))^2 - De (Eq. 6); excited surface
 * A + B exp(-beta (r - rc)) (Eq. 7 is A = 0, B = 2 D_e); constant
 * transition dipole d [e a0]; absorbing mask cos(pi/2 (r-ra)/(rmax-ra))^p
 * for r > ra (ra >= rmax disables it).
 *
 * An R-dependent transition dipole (dipole_R) acts point-wise along R in the
 * coupling, exp(i dtau d(R) sigma_x (x) E'.R^), and in the dipole,
 * 2 Re sum_R d(R) chi_g^dagger R^ chi_e dR; the dipole is then read from
 * psi = T^{1/2} s by one more kernel per molecular step.  It needs jmax <= 4,
 * nr 64 or 128 and the full state (the point-resident kernels; the fused
 * layout at nr 128 only), else MS_EUNSUPPORTED; non-finite values give
 * MS_EINVAL.
 *
 * MS_MODEL_BLOCH (the frozen molecules of the scaling-experiments section,
 * Fig. 5d): a two-level emitter with its ro-vibrational degrees of freedom
 * frozen, H = w0 |e><e| - d (n . E)(|g><e| + |e><g|), transition energy
 * bloch_w0_eV >= 0, transition dipole dipole_ea0 along the molecule frame's
 * z axis n, optional population relaxation and dephasing times bloch_T1_s,
 * bloch_T2_s >= 0 (0 = none).  The Bloch vector (u, v, w) = (2 Re rho_eg,
 * 2 Im rho_eg, rho_ee - rho_gg) starts at (0, 0, -1) and takes one RK4 step
 * per molecular step with the field held at E^n; the dipole is d u along n.
 * morse_re is the frozen bond length (Eq. 8 readout: numerator re P_e,
 * denominator P_e); the other fields are ignored, and the mol_path,
 * precision and state_form options do not apply to it (its state is three
 * FP64 numbers per molecule). */
enum { MS_MODEL_WAVEPACKET = 0, MS_MODEL_BLOCH = 1 };
typedef struct {
  int32_t nr, jmax;
  double rmin, rmax, mass_me;
  double morse_De, morse_a, morse_re;
  double exc_A, exc_B, exc_beta, exc_rc;
  double dipole_ea0;
  double absorber_r, absorber_power;
  int32_t model;              /* MS_MODEL_WAVEPACKET or MS_MODEL_BLOCH */
  double bloch_w0_eV;         /* MS_MODEL_BLOCH: transition energy */
  double bloch_T1_s, bloch_T2_s;  /* MS_MODEL_BLOCH: relaxation times, 0 = none */
  const double* dipole_R;     /* MS_MODEL_WAVEPACKET: NULL for the constant dipole_ea0, or an
                                 R-dependent transition dipole d(R) at the nr grid points
                                 (e a0), copied; see below */
} ms_species;

/* Molecules: species_id, sim_id [n]; pos_m [n][3] absolute position in the
 * sim's box (metres; cell = floor(pos/dx), a point on a face belongs to
 * the upper cell); orient [n][4] unit quaternion (w,x,y,z) rotating the
 * molecule frame into the lab frame.  Every molecule starts in the v=0,
 * j=0, m=0 state of the ground surface. */
typedef struct {
  int32_t n_species;
  const ms_species* species;
  int64_t n_molecules;
  const int32_t* species_id;
  const int32_t* sim_id;
  const double* pos_m;
  const double* orient;
} ms_molecules_desc;

/* Options.  alloc/free: optional device allocator (e.g. a framework's
 * caching allocator); when NULL the library uses cudaMalloc/cudaFree.
 * stream: cudaStream_t to run on; NULL = a stream the library creates. */
typedef struct {
  int32_t precision;    /* MS_PREC_FP32 or MS_PREC_MIXED_F16X3 */
  int32_t mol_substeps; /* N: the molecules advance on field steps n with
                           n % N == 0, by a step of N dt, under E^n; their
                           dipole change enters that step's E update (Sec. 2's
                           multiscale cadence).  0 means 1; 1..65536, else
                           MS_EINVAL. */
  int32_t drive;        /* MS_DRIVE_FDTD or MS_DRIVE_PRESCRIBED */
  void* (*alloc)(size_t bytes, void* ctx);
  void (*free)(void* ptr, void* ctx);
  void* alloc_ctx;
  void* stream;
  int32_t mol_path;     /* MS_MOL_AUTO, MS_MOL_FUSED or MS_MOL_STREAMING */
  int32_t state_form;   /* MS_STATE_FULL or MS_STATE_PARITY */
  int32_t step_graphs;  /* MS_GRAPHS_AUTO or MS_GRAPHS_OFF (see ms_step) */
  int32_t autotune;     /* MS_TUNE_OFF or MS_TUNE_MEASURE (see MS_KERN_*) */
} ms_options;

/* Create a simulation: validates the descriptors, builds the species
 * tables (potential and kinetic phases, angular coupling matrices, Fourier
 * grid ground state), sorts molecules by cell, allocates and uploads.
 * On failure *out is NULL and nothing is leaked. */
ms_status ms_create(const ms_grid_desc* grid, const ms_materials_desc* materials,
                    const ms_molecules_desc* molecules, const ms_options* opts,
                    ms_sim** out);

/* Advance n coupled steps (n >= 0) on the handle's stream, asynchronously.
 * Step order: H update, molecular step under E^n, polarization change,
 * E update (the paper's leap-frog with the molecular current).  With
 * MS_GRAPHS_AUTO the launches of whole cycles replay from a CUDA graph
 * captured on first use (and again after ms_set_prescribed_field,
 * ms_set_replay_field or ms_set_detectors change what the kernels read). */
ms_status ms_step(ms_sim* sim, int64_t n);

/* Allocation-free stepping.  The paper has no counterpart: this is a library
 * service.  It advances n steps exactly like ms_step, but species run in the
 * streaming form (MS_MOL_STREAMING) take the scratch that holds (T - 1)s from
 * a fixed 64 MiB device array compiled into the library instead of from the
 * handle's buffer; the call itself allocates nothing (no cudaMalloc, no
 * allocator callback, no library routine that allocates).  It is meant for
 * callers that cannot allocate device memory at the point where they step:
 * for instance, code that runs inside a fixed memory arena or under a
 * budget that forbids new device allocations.
 *   - Limit: each streaming species takes its own region of the array,
 *     n_molecules * 2 (jmax+1)^2 * nr * 8 bytes rounded up to 256 bytes
 *     (half the rows for MS_STATE_PARITY), and the regions of all of a
 *     handle's streaming species together must fit in 64 MiB; otherwise
 *     MS_EINVAL is returned before anything is launched.
 *   - The array is shared by every call and every handle in the process, on
 *     each device; it keeps the last call's contents, and each step rewrites
 *     the part it reads before reading it.  Calls whose work overlaps on the
 *     GPU (different streams or threads) race on it: serialise them.
 *   - Every GPU that loads the library holds the 64 MiB until the process
 *     exits.  ms_create looks the array's address up with the handle's
 *     device current (this may load the library's device code on that device
 *     and so take the 64 MiB then); if that lookup fails, ms_step_noalloc
 *     returns MS_ECUDA.  Stepping a handle with ms_step and ms_step_noalloc
 *     in any order gives the same results.
 * Errors as for ms_step. */
ms_status ms_step_noalloc(ms_sim* sim, int64_t n);

/* Number of steps taken so far. */
int64_t ms_step_count(const ms_sim* sim);

/* Copy the E (which = MS_FIELD_E) or H field of one sim to host_dst,
 * 3 * nz*ny*nx floats: all x components, then y, then z, in the Yee
 * positions of the header's layout note (the fields of Eq. 1 as the FDTD
 * section stores them).  n is the capacity of host_dst in floats; MS_EINVAL
 * for a smaller n, a bad `which` or sim, or a handle without a field grid.
 * Synchronous. */
ms_status ms_read_fields(ms_sim* sim, int32_t which, int32_t sim_index, float* host_dst,
                         size_t n);

/* Overwrite the E or H field of one sim (same layout and errors as
 * ms_read_fields); sets the initial or a test field of Eq. 1's leap-frog.
 * Synchronous; src is copied. */
ms_status ms_write_fields(ms_sim* sim, int32_t which, int32_t sim_index, const float* src,
                          size_t n);

/* Per-molecule populations P_g, P_e (FP64) of molecules [first, first+count)
 * in the caller's molecule order, at the current time: the norms
 * sum_{j,m} integral |xi^{g,e}_{jm}(R)|^2 dR of the two surfaces' wavepackets
 * of Eq. 3 (for frozen two-level molecules, rho_gg and rho_ee).  Either
 * output may be NULL.  MS_EINVAL for a range outside the molecules. */
ms_status ms_read_populations(ms_sim* sim, int64_t first, int64_t count, double* Pg,
                              double* Pe);

/* Per-molecule dissociation observables (FP64): norm removed by the
 * absorber since t=0 on each surface, and the numerator <chi_e|R|chi_e>
 * and denominator <chi_e|chi_e> of Eq. 8 at the current time.  Any output
 * may be NULL. */
ms_status ms_read_dissociation(ms_sim* sim, int64_t first, int64_t count, double* absorbed_g,
                               double* absorbed_e, double* R_e_num, double* R_e_den);

/* Per-molecule lab-frame induced dipole (a.u., FP64, [count][3]) at the
 * current time: the expectation value of the transition dipole between the
 * two surfaces' wavepackets (Eq. 4's coupling operator), rotated from the
 * molecule frame to the lab frame; the dipole density that enters Eq. 1's
 * polarization current is this divided by the cell volume.  MS_EINVAL for a
 * NULL mu or a range outside the molecules. */
ms_status ms_read_dipoles(ms_sim* sim, int64_t first, int64_t count, double* mu);

/* Prescribed drive (MS_DRIVE_PRESCRIBED): molecule k sees the lab field
 * amp[k][0..2] * wave[n] (V/m) during step n; the field grid is not
 * advanced.  nsteps samples of wave; ms_step fails with MS_EINVAL beyond
 * them. */
ms_status ms_set_prescribed_field(ms_sim* sim, const float* amp, const float* wave,
                                  int64_t nsteps);

/* Replay drive (MS_DRIVE_PRESCRIBED): molecule k sees the lab field
 * E[n][k][0..2] (V/m) during step n, for nsteps steps; E is
 * [nsteps][n_molecules][3] FP32 in the caller's molecule order, copied.
 * It replaces any amp/wave drive set before, and a later
 * ms_set_prescribed_field replaces it.  Fields recorded on a coupled run by
 * ms_record_local_fields replay that run's molecular dynamics exactly
 * (same arithmetic on the same FP32 inputs).  Errors: MS_EINVAL for a NULL
 * argument, nsteps <= 0 or an FDTD-driven handle; MS_ENOMEM. */
ms_status ms_set_replay_field(ms_sim* sim, const float* E, int64_t nsteps);

/* Advances nsteps coupled steps (as ms_step) and records, at every step n,
 * the lab-frame E^n that drives each listed molecule: the components owned
 * by its cell (the gather of the coupled step, Eq. 1 grid, in V/m).  dst is
 * [nsteps][m][3] FP32, caller-owned, written when the call returns
 * (synchronous).  mol_ids: m molecule indices in the caller's order.
 * Errors: MS_EINVAL (NULL pointer, m <= 0, nsteps < 0, an index out of
 * range, or a handle without a field grid), MS_ENOMEM for the temporary
 * device buffer, and the latched errors of ms_step. */
ms_status ms_record_local_fields(ms_sim* sim, const int64_t* mol_ids, int64_t m, float* dst,
                                 int64_t nsteps);

/* Spectral detection (the transmission / reflection spectra of Figs. 2, 4
 * and 6a): running discrete Fourier transforms of the tangential fields on
 * z-planes, accumulated every step from the next ms_step on.
 *   - Accumulator: F^(omega) = dt sum_n F(t_n) e^{i omega t_n}, FP64, per
 *     cell, with Ex, Ey on plane k at t_{n+1} and Hx, Hy averaged over the
 *     planes k -+ 1/2 at t_{n+1/2}; so Ex with Hy and Ey with Hx share their
 *     in-plane positions.
 *   - planes_z: nplanes (1..16) absolute z indices in [1, nz - 1).
 *   - omega: nfreq (1..512) angular frequencies in rad/s.
 * A call replaces the detectors set before and zeroes the accumulators;
 * each call allocates their device memory (nsim * nplanes * nfreq * 4 * nx
 * * ny * 16 bytes) until ms_destroy.  FDTD-driven handles only.  Errors:
 * MS_EINVAL, MS_ENOMEM. */
ms_status ms_set_detectors(ms_sim* sim, const int32_t* planes_z, int32_t nplanes, const double* omega,
                           int32_t nfreq);

/* Poynting flux spectrum through detector plane `plane` (in +z):
 * flux[s][f] = Re sum_cells (Ex^ conj(Hy^) - Ey^ conj(Hx^)) dx^2 for
 * simulation s and frequency f ([nsim][nfreq], FP64, in J s: the
 * accumulators carry dt).  The energy through the plane is
 * (1/pi) integral_0^inf flux d omega.  Synchronous. */
ms_status ms_read_flux(ms_sim* sim, int32_t plane, double* flux);

/* Raw accumulator of plane `plane`, simulation `sim`, component (0 Ex, 1 Ey,
 * 2 Hx, 3 Hy) and frequency index `freq`: [ny][nx] complex FP64 as
 * (re, im) pairs into dst (2 ny nx doubles).  Synchronous. */
ms_status ms_read_dft(ms_sim* sim, int32_t plane, int32_t sim_index, int32_t component, int32_t freq,
                      double* dst);

/* Checkpoint / resume (no counterpart in the paper, which runs to completion).
 * ms_save writes the whole evolving state to the file `path`:
 *   - the fields E and H;
 *   - the Drude current;
 *   - the CPML auxiliaries and the incident line;
 *   - every species' wavepackets (Bloch vectors for frozen molecules);
 *   - the molecules' dipoles, populations, absorbed norm and rounding
 *     feedback factors;
 *   - the detectors' running Fourier transforms (when set);
 *   - the step counter.
 * The inputs (geometry, materials, molecules, drive samples) are not saved.
 * ms_load restores such a file into a handle created from the same
 * descriptors and options; the sizes, the sub-step count and the source
 * kind in the file must match (MS_EINVAL otherwise).  A prescribed or replay
 * drive is set again by the caller.  N steps equal N/2 steps, save, load
 * into a fresh handle, N/2 steps, bit for bit.  Both calls are synchronous
 * and stage through two pinned 64 MiB host buffers (pageable memory when
 * pinned memory cannot be had).  Errors:
 * MS_EINVAL (NULL argument, size mismatch), MS_EIO (open, short read or
 * write, wrong magic or version), MS_ECUDA. */
ms_status ms_save(ms_sim* sim, const char* path);
ms_status ms_load(ms_sim* sim, const char* path);

/* Phase timing with CUDA events on the handle's stream.  Between
 * ms_timing_begin and ms_timing_end every ms_step records events around its
 * phases; ms_timing_end synchronises and writes the summed durations in
 * milliseconds: out[0] H half step (H update and incident line), out[1]
 * molecular step (all species), out[2] E half step (E update, incident
 * line, spectral detection when set), out[3] their sum (the one-thread step
 * counter runs between steps, outside these spans), out[4] the molecular
 * step's first stage (streaming form: field records and kinetic pass),
 * out[5] its second stage (streaming form: R-space pass; fused form: the
 * whole step); *steps receives the number of steps timed and *launches the
 * number of kernels launched.  While timing is on, ms_step launches every
 * kernel itself (no graph replay).  Errors: MS_EINVAL for a NULL handle or
 * out, MS_ECUDA. */
ms_status ms_timing_begin(ms_sim* sim);
ms_status ms_timing_end(ms_sim* sim, double out[6], int64_t* steps, int64_t* launches);

/* Diagnostic of the bounded waits (no counterpart in the paper).  The
 * molecular kernels wait for their bulk copies with a bounded wait: each
 * try suspends the thread until the copy lands or a time hint expires, and
 * after the last try the kernel records MS_ETIMEOUT and returns instead of
 * hanging.  This runs that routine in one CTA on a barrier that nothing
 * completes, with `tries` (1..100000) tries of up to 10 us, so the wait runs
 * out.  Expected result: MS_ETIMEOUT, with the device context still usable.
 * MS_EINVAL for tries out of range, MS_ENOMEM / MS_ECUDA on runtime errors.
 * Needs no handle; allocates one int of device memory. */
ms_status ms_check_bounded_wait(int32_t tries);

/* The molecular kernel layout a species runs in (MS_MOL_FUSED or
 * MS_MOL_STREAMING, after MS_MOL_AUTO resolved it; a MS_MODEL_BLOCH species
 * reports MS_MOL_FUSED: one kernel reads and writes its state once per step);
 * MS_EINVAL for a NULL handle or a species index out of range. */
int32_t ms_species_path(const ms_sim* sim, int32_t species);

/* The plan of a species (see MS_KERN_*): layout, kernel and chunk width (0
 * where the kernel has none or follows its rule).  MS_EINVAL for a NULL
 * handle or pointer or a species index out of range. */
ms_status ms_species_plan(const ms_sim* sim, int32_t species, int32_t* path, int32_t* kernel, int32_t* chunk);

/* Pin a species' plan: one of the plans it can run (MS_EINVAL otherwise,
 * nothing changed); kernel MS_KERN_DEFAULT restores the static rule for the
 * given layout.  A switch to the streaming layout allocates its (T - 1)s
 * scratch (MS_ENOMEM if that fails).  Takes effect from the next step. */
ms_status ms_set_species_plan(ms_sim* sim, int32_t species, int32_t path, int32_t kernel, int32_t chunk);

/* Pipelined molecular step (no counterpart in the paper; a scheduling
 * choice).  batches = 0 (the default): the molecular step runs stage 1 (the
 * frame-field records and the kinetic pass) of every species, then stage 2
 * (the R-space pass) of every species, on the handle's stream.  batches = n
 * >= 1: every streaming-layout species is cut into n runs of consecutive
 * molecules (other species: one run each); stage 1 of each run is issued on
 * the handle's stream and stage 2 of the same run on a second stream after
 * it, so the kinetic pass of run k + 1 (bound by HBM bandwidth) can execute
 * while the R-space pass of run k (bound by the SMs' shared-memory pipe)
 * does; the handle's stream waits for the last run before the E half step.
 * Runs hold disjoint molecules and every molecule gets the same kernels on
 * the same data, so results are identical bit for bit for every n.  With
 * n >= 1 the phase timing (ms_timing_begin) reports the molecular step as a
 * whole: stage 1's phase then holds all of it and stage 2's is empty.
 * Takes effect from the next
 * step.  MS_EINVAL for a NULL handle or batches outside 0..16; MS_ECUDA if
 * the second stream or its events cannot be created. */
ms_status ms_set_mol_batches(ms_sim* sim, int32_t batches);
/* The handle's batches (ms_set_mol_batches); -1 for a NULL handle. */
int32_t ms_mol_batches(const ms_sim* sim);

/* Extended plan (no counterpart in the paper): plan[0] layout, plan[1]
 * kernel, plan[2] chunk, as for ms_species_plan, and plan[3] the grid of the
 * persistent tiled kernels (MS_KERN_TILE, MS_KERN_PAIR): resident CTAs per SM (1..32, fewer
 * if fewer fit), so each CTA walks about n_molecules / (plan[3] x SMs)
 * molecules; 0 = as many CTAs as fit at once; -1 = one CTA per molecule.
 * Other kernels take plan[3] = 0.  Every grid computes each molecule with the
 * same arithmetic, so results are identical bit for bit; the autotuner
 * (MS_TUNE_MEASURE) times the grids with the tile widths.  Setting a plan as
 * ms_set_species_plan does, plus the grid; ms_set_species_plan sets grid 0.
 * MS_EINVAL for a NULL handle or plan, a species out of range, a grid out of
 * range or given to another kernel, or a plan the species cannot run. */
ms_status ms_species_plan_ex(const ms_sim* sim, int32_t species, int32_t plan[4]);
ms_status ms_set_species_plan_ex(ms_sim* sim, int32_t species, const int32_t plan[4]);

/* Device memory held by the simulation, in bytes. */
size_t ms_device_bytes(const ms_sim* sim);

/* Release the handle: waits for its stream, frees every device block (through
 * the caller's allocator when one was given), destroys the library's own
 * stream and any captured graph.  NULL is a no-op. */
void ms_destroy(ms_sim* sim);

/* A static, NUL-terminated description of a status code ("unknown status" for
 * a value that is not one). */
const char* ms_status_string(ms_status s);

#ifdef __cplusplus
}
#endif
#endif /* MS_H */
