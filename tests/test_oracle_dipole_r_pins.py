"""Pins of the oracle's R-dependent transition dipole d(R) (the NEXT row of
the parity-reduced state: a dipole that varies with the bond length).  The
step and the dipole are checked against dense brute-force operators built
independently with scipy's matrix exponential on a small grid, and the
constant table against the constant dipole."""
import dataclasses

import numpy as np
import pytest
import scipy.linalg as sla

import workloads as W
from oracle.constants import F_AU
from oracle.molecule import SpeciesEnsemble, angular_matrices, kinetic_propagator, mask, potentials, \
    radial_grid, channels


def _species(nr=16, jmax=1, dR=None):
    sp = W.Species(nr=nr, jmax=jmax, A=0.05, absorber_r=8.0)
    if dR is not None:
        sp = dataclasses.replace(sp, dipole_R=tuple(dR))
    return sp


def _d_table(sp):
    r, _ = radial_grid(sp)
    return 0.6 + 0.5 * np.tanh(r - 3.0) + 0.2 * np.exp(-(r - 2.2) ** 2)


def test_step_matches_dense_brute_force():
    """One split-operator step with d(R) equals T^1/2 Mask V^1/2 expm(i dtau
    d(R) sigma_x (x) M) V^1/2 T^1/2 assembled as dense matrices over
    (surface, channel, R)."""
    sp0 = _species()
    dtab = _d_table(sp0)
    sp = _species(dR=dtab)
    rng = np.random.default_rng(3)
    q = rng.standard_normal((1, 4))
    dtau = 0.4
    ens = SpeciesEnsemble(sp, q, dtau)
    # a random normalised starting state (not the ground state)
    psi0 = rng.standard_normal(ens.psi.shape) + 1j * rng.standard_normal(ens.psi.shape)
    psi0 /= np.sqrt((np.abs(psi0) ** 2).sum() * ens.dR)
    ens.psi = psi0.copy()
    E = np.array([[2.0e10, -1.0e10, 3.0e10]])
    ens.step(E)

    nrot, nr = ens.nrot, sp.nr
    r, dRr = radial_grid(sp)
    X, Y, Z = angular_matrices(sp.jmax)
    O = ens.O[0]
    Em = O.T @ E[0] / F_AU
    M = Em[0] * X + Em[1] * Y + Em[2] * Z
    sx = np.array([[0, 1], [1, 0]])
    Kgen = np.kron(np.kron(sx, M), np.diag(dtab))           # sigma_x (x) M (x) d(R)
    K = sla.expm(1j * dtau * Kgen)
    Ug, Ue = potentials(sp, r)
    jj = np.array([j * (j + 1) for j, _ in channels(sp.jmax)], float)
    V = np.stack([Ug[None] + jj[:, None] / (2 * sp.mass * r ** 2), Ue[None] + jj[:, None] / (2 * sp.mass * r ** 2)])
    Vh = np.diag(np.exp(-0.5j * dtau * V.ravel()))
    Th = np.kron(np.eye(2 * nrot), kinetic_propagator(sp, 0.5 * dtau))
    Mk = np.diag(np.tile(mask(sp), 2 * nrot))
    step = Th @ Mk @ Vh @ K @ Vh @ Th
    want = (step @ psi0.ravel()).reshape(ens.psi.shape)
    assert np.abs(ens.psi - want).max() < 1e-12


def test_dipole_matches_dense_expectation():
    """mu' = <psi| sigma_x (x) A (x) d(R) |psi> dR for A = X, Y, Z."""
    sp = _species(dR=_d_table(_species()))
    rng = np.random.default_rng(4)
    ens = SpeciesEnsemble(sp, np.array([[1.0, 0, 0, 0]]), 0.1)
    psi = rng.standard_normal(ens.psi.shape) + 1j * rng.standard_normal(ens.psi.shape)
    X, Y, Z = angular_matrices(sp.jmax)
    sx = np.array([[0, 1], [1, 0]])
    v = psi.ravel()
    for c, A in enumerate((X, Y, Z)):
        D = np.kron(np.kron(sx, A), np.diag(ens.d_r))
        want = (v.conj() @ D @ v).real * ens.dR
        assert abs(ens.dipole_mol(psi)[0, c] - want) < 1e-12 * max(1.0, abs(want))


def test_constant_table_equals_constant_dipole():
    sp = _species(jmax=2)
    spt = dataclasses.replace(sp, dipole_R=tuple(np.full(sp.nr, sp.dipole)))
    q = np.random.default_rng(5).standard_normal((3, 4))
    a, b = SpeciesEnsemble(sp, q, 0.2), SpeciesEnsemble(spt, q, 0.2)
    E = np.random.default_rng(6).standard_normal((3, 3)) * 3e10
    for _ in range(20):
        ma, mb = a.step(E), b.step(E)
    assert np.array_equal(a.psi, b.psi) and np.array_equal(ma, mb)


def test_norm_conserved_with_dR():
    sp = _species(jmax=2, dR=_d_table(_species(jmax=2)))
    sp = dataclasses.replace(sp, absorber_r=sp.rmax)       # no absorber
    ens = SpeciesEnsemble(sp, np.random.default_rng(7).standard_normal((2, 4)), 0.3)
    E = np.random.default_rng(8).standard_normal((2, 3)) * 5e10
    for _ in range(50):
        ens.step(E)
    assert np.abs(ens.populations().sum(axis=1) - 1.0).max() < 1e-12
    assert ens.populations()[:, 1].max() > 1e-4
