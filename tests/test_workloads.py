"""The seeded input recipes (no GPU): what the generators draw is what the benchmark and the
tests claim they draw.

The batched uneven workload: nx ~ U{4..24}, nu ~ U{2..8}, N ~ U{50..500}; every stage's A_k has
its spectral radius in [0.9, 1.05] (the signed-permutation similarity keeps the base matrix's
eigenvalues); B_k and the disturbances e_k ~ U[-0.3, 0.3] per stage; Q = I, R = 0.1 I,
|u| <= 1, |x| <= 5, x0 ~ U[-3, 3], zero reference, rho = 1. The large-state workload: nx 48,
nu 16, A with spectral radius 0.95, the calibrated input bound. Same seed, same arrays.
"""
import numpy as np

from paper_2601_14414_gb300 import workloads as W


def test_batched_uneven_recipe():
    insts = W.batched_uneven(seed=3, batch=48)
    nxs, nus, Ns = W.batched_dims(seed=3, batch=48)
    for j, inst in enumerate(insts):
        nx, nu, N = inst["nx"], inst["nu"], inst["N"]
        assert (nx, nu, N) == (nxs[j], nus[j], Ns[j])
        assert 4 <= nx <= 24 and 2 <= nu <= 8 and 50 <= N <= 500 and not inst["lti"]
        assert inst["A"].shape == (N, nx, nx) and inst["B"].shape == (N, nx, nu)
        assert inst["e"].shape == (N, nx) and np.all(np.abs(inst["e"]) <= 0.3)
        radii = np.max(np.abs(np.linalg.eigvals(inst["A"])), axis=1)
        assert np.all(radii >= 0.9 - 1e-9) and np.all(radii <= 1.05 + 1e-9), j
        np.testing.assert_array_equal(inst["q"], np.ones(nx))
        np.testing.assert_array_equal(inst["r"], 0.1 * np.ones(nu))
        np.testing.assert_array_equal(inst["xmax"], 5.0 * np.ones(nx))
        np.testing.assert_array_equal(inst["umax"], np.ones(nu))
        np.testing.assert_array_equal(inst["xmin"], -inst["xmax"])
        np.testing.assert_array_equal(inst["umin"], -inst["umax"])
        assert np.all(np.abs(inst["x0"]) <= 3.0) and inst["rho"] == 1.0
        assert not np.any(inst["ref"])


def test_batched_uneven_dims_cover_the_ranges():
    nxs, nus, Ns = W.batched_dims(seed=3, batch=4096)
    assert (nxs.min(), nxs.max(), nus.min(), nus.max()) == (4, 24, 2, 8)
    assert Ns.min() >= 50 and Ns.max() <= 500
    assert 1.05e6 < int(np.sum(Ns)) < 1.2e6          # about 1.13M stages


def test_generators_are_seeded():
    a, b = W.batched_uneven(seed=7, batch=3), W.batched_uneven(seed=7, batch=3)
    c = W.batched_uneven(seed=8, batch=3)
    for x, y in zip(a, b):
        for key in ("A", "B", "e", "x0"):
            np.testing.assert_array_equal(x[key], y[key])
    assert any(x["nx"] != y["nx"] or not np.array_equal(x["x0"], y["x0"]) for x, y in zip(a, c))


def test_large_state_recipe():
    insts = W.large_lti(batch=2)
    for inst in insts:
        assert (inst["nx"], inst["nu"], inst["N"], inst["lti"]) == (48, 16, 1000, True)
        radius = np.max(np.abs(np.linalg.eigvals(inst["A"])))
        assert abs(radius - 0.95) < 1e-9
        assert np.all(np.abs(inst["e"]) <= 0.3)
        np.testing.assert_array_equal(inst["umax"], W.LARGE_LTI_UMAX * np.ones(16))
        assert np.all((inst["q"] >= 0.1) & (inst["q"] <= 10.0))
        assert np.all((inst["r"] >= 0.01) & (inst["r"] <= 1.0))


def test_plain_lti_recipe():
    inst = W.plain_lti()
    assert (inst["nx"], inst["nu"], inst["N"]) == (4, 2, 20)
    assert abs(np.max(np.abs(np.linalg.eigvals(inst["A"]))) - 0.95) < 1e-12
    np.testing.assert_array_equal(inst["r"], 0.1 * np.ones(2))
