"""The seeded input generators: deterministic, in range, shaped like the
paper's workloads (split rings, triangular nanoholes, a molecular layer)."""
import numpy as np

import workloads as W


def test_config0_is_deterministic_and_in_layer():
    a, b = W.config0(), W.config0()
    assert np.array_equal(a.pos, b.pos) and np.array_equal(a.quat, b.quat)
    k = np.floor(a.pos[:, 2] / a.dx)
    assert k.min() >= 40 and k.max() <= 43
    assert a.n_molecules == 1000 and a.mat_id.max() == 0
    assert np.allclose(np.linalg.norm(a.quat, axis=1), 1.0)


def test_srr_and_nanohole_geometry():
    wl = W.config1(n_molecules=10)
    m = wl.mat_id[0]
    ring = m[55] == W.configs.MAT_SILVER
    # 30x30 outer square minus 10x10 hole minus a 5x10 gap
    assert ring.sum() == 30 * 30 - 10 * 10 - 5 * 10
    assert (m[70] == W.configs.MAT_GLASS).all()
    wl4 = W.config4(n_per_sim=10, nsim=2)
    film = wl4.mat_id[0, 40] == W.configs.MAT_SILVER
    hole = (~film).sum()
    side = 42.0
    assert abs(hole - side * side * np.sqrt(3) / 4) < 0.08 * hole
    assert wl4.src.shape == (2, 4) and wl4.src[1, 1] == 2.4


def test_config2_cells_are_distinct():
    wl = W.custom("distinct", 64, 64, 64, layer=(40, 42), n_per_sim=5000, distinct=True)
    c = np.floor(wl.pos / wl.dx).astype(int)
    lin = (c[:, 2] * 64 + c[:, 1]) * 64 + c[:, 0]
    assert np.unique(lin).size == 5000
