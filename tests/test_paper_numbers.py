"""Host-side helpers checked against numbers the paper prints (tests/golden)."""
import json
import os

import pytest

from paper_2308_16597_gb300 import metrics

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_numbers.json")))


@pytest.mark.parametrize("row", GOLD["mlups"])
def test_mlups_definition_reproduces_table_1(row):
    v = metrics.mlups(row["nx"], row["ny"], row["steps"], row["seconds"])
    assert abs(v - row["mlups"]) / row["mlups"] < 2e-3


@pytest.mark.parametrize("row", GOLD["volume_fraction"])
def test_volume_fractions(row):
    v = metrics.volume_fraction(row["n"], row["d_mm"] * 0.1, row["W_cm"], row["H_cm"])
    assert abs(v - row["phi"]) < 6e-4


@pytest.mark.parametrize("row", GOLD["rep_ar"])
def test_reynolds_archimedes_relation(row):
    assert abs(metrics.reynolds_from_archimedes(row["Ar"]) - row["Re_p"]) / row["Re_p"] < 2e-3


@pytest.mark.parametrize("row", GOLD["viscosity_units"])
def test_lattice_viscosity_conversion(row):
    v = metrics.lattice_viscosity(row["nu_phys"], row["t_star"], row["l_star"])
    assert abs(v - row["nu_lu"]) < 1e-12


def test_zone_size_of_the_paper_particles(orc):
    z = GOLD["zone"]
    assert orc.zone_size(z["d_lu"] / 2) == z["N"]
    assert orc.slot_capacity(z["d_lu"] / 2) == z["capacity"]


def test_parallel_efficiency():
    e = GOLD["parallel_efficiency"]
    assert abs(metrics.parallel_efficiency(e["mlups_n"], e["mlups_1"], e["n"]) - e["efficiency"]) < 1e-3


def test_bytes_per_update():
    assert metrics.bytes_per_update(4) == 112 and metrics.bytes_per_update(2) == 56
