"""FP64 CPU oracle for the coupled Maxwell-Schroedinger step (arXiv 2209.04487).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
``bench.py``'s CPU-baseline / reference legs may import or run this package.
The product library never calls it, links it or falls back to it.

It is a plain, slow, literal restatement of the paper's equations in float64
NumPy, sharing no code with the CUDA path (the seeded input generators in
``workloads/`` are the only common module):

* ``fdtd``     -- Yee leap-frog for Eq. 1, Drude current Eq. 2, CPML in z,
                  periodic x/y, TF/SF plane-wave source.
* ``molecule`` -- Eqs. 3-7: rotational expansion, coupled two-surface TDSE,
                  effective Hamiltonians, split-operator propagation,
                  dipole / population / absorbed-norm / Eq. 8 observables.
* ``coupled``  -- the coupled time step (fields drive molecules, the
                  molecular polarization current feeds back into Ampere's law),
                  with the every-N-th-step molecular cadence.
* ``bloch``    -- frozen two-level molecules (Bloch equations, RK4; the
                  scaling-experiments section, Fig. 5d).
* ``spectra``  -- running DFTs on z-planes and Poynting flux spectra (the
                  transmission / reflection spectra of Figs. 2, 4 and 6a).

Every function cites the passage of the paper it follows.  Functions whose
result has no independent check carry the words "parity unpinned".
"""
