"""Host arithmetic of the final observables (Section 2.2), checked on the oracle's outputs."""
import math

import numpy as np

import oracle as O
from paper_1208_0166_gb300 import observables as obs
from paper_1208_0166_gb300.workloads import random_angles
from tests import lattice_np as ln


def test_static_potential_of_an_area_law():
    Nt, sigma = 8, 0.2
    r = np.arange(1, 5)
    corr = np.exp(-sigma * r * Nt) + 0j
    assert np.allclose(obs.static_potential(corr, Nt), sigma * r)
    assert math.isnan(obs.static_potential(np.array([-1e-9]), Nt)[0])


def test_uniform_background_field_has_no_connected_part():
    """A uniform field is the same with and without sources: the connected average vanishes."""
    L, Nt = 4, 4
    th, E, B = ln.constant_field(L, Nt, 1, 1)
    ml = O.Lattice(L, Nt, 1.0, 1, theta=th).multilevel(2, 2, 2, d_max=1, sub_metro=0, sub_or=0)
    assert np.max(np.abs(obs.connected(ml["fields"], ml["corr"], ml["vac"]))) < 1e-13
    comp = obs.field_components(ml["fields"], ml["corr"], ml["vac"], 1.0)
    assert np.max(np.abs(comp["E_x"])) < 1e-13


def test_connected_average_definition_on_a_frozen_configuration():
    L, Nt = 4, 4
    lat = O.Lattice(L, Nt, 1.0, 1, theta=random_angles(L, Nt, 7))
    ml = lat.copy().multilevel(2, 1, 2, d_max=1, sub_metro=0, sub_or=0)
    conn = obs.connected(ml["fields"], ml["corr"], ml["vac"])
    # element by element: Re(<P*P O>/<P*P>) - <O>
    for r in range(2):
        for d in range(2):
            for ch in range(8):
                want = (ml["fields"][r, d, ch] / ml["corr"][r]).real - ml["vac"][ch]
                assert abs(conn[r, d, ch] - want) < 1e-15
    comp = obs.field_components(ml["fields"], ml["corr"], ml["vac"], 0.81)
    assert np.allclose(comp["B_x"], 0.9 * conn[:, :, 6])
    assert np.allclose(comp["E_y^2"], -0.81 * conn[:, :, 3])
