"""The seeded input generator (no exact-exchange arithmetic): the host-side
subset of orbitals used by the CPU baseline and the reference arm equals the
corresponding rows of the full generator, and the orbitals are orthonormal in
the discrete inner product h^3 sum_m."""

import numpy as np
import pytest

from paper_1712_07973_gb300 import synth


@pytest.mark.parametrize("recipe", [
    synth.OrbitalRecipe(n=20, h=0.4, norb=9, nsites=5, seed=3, gauss_per_orb=4, sigma=(0.7, 1.8),
                        p_type=True),
    synth.OrbitalRecipe(n=16, h=0.5, norb=7, nsites=8, seed=1, gauss_per_orb=3, lattice=2.0),
])
def test_orbital_subset_equals_full_generator(recipe):
    full = synth.make_orbitals(recipe)
    idx = [0, 3, recipe.norb - 1]
    sub = synth.orbital_subset(recipe, idx, chunk=8)
    assert np.max(np.abs(sub - full[idx])) <= 1e-13 * np.max(np.abs(full))


def test_orbitals_are_orthonormal():
    r = synth.OrbitalRecipe(n=24, h=0.45, norb=6, nsites=4, seed=9, gauss_per_orb=5,
                            sigma=(0.7, 1.5), p_type=True)
    psi = synth.make_orbitals(r).reshape(r.norb, -1)
    S = r.h ** 3 * psi @ psi.T
    assert np.max(np.abs(S - np.eye(r.norb))) <= 1e-12


def test_batched_workloads_are_seeded():
    a = [(x.n, x.norb, x.seed) for x in synth.small_batched_workload()]
    b = [(x.n, x.norb, x.seed) for x in synth.small_batched_workload()]
    assert a == b and len(a) == 64
    assert all(x[0] in (32, 40, 48) and 8 <= x[1] <= 24 for x in a)
