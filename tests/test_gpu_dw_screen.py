"""Density-weighted screening of the SCF's incremental builds (fsim_scf_opts.dw_screen).

An increment G(dD) may skip the quartets with Q_ab Q_cd max|dD| < tau, the
same bound that ordinary Schwarz screening gives a full build; the
FP64-accurate resets are full builds at the plain threshold.  The converged
energy must therefore agree with the unscreened run's, and with the
oracle's, to the SCF tolerance used elsewhere (1e-8 Eh), while the
increments evaluate fewer quartets.
"""
import json
import os

import numpy as np
import pytest

from fsim_synth import workload

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2510_24968_gb300.build import build
    build()
    yield


@pytest.mark.parametrize("name", ["water4", "water8"])
def test_dw_screened_scf_same_energy_fewer_quartets(name):
    from paper_2510_24968_gb300 import FSIM_MIXED, Basis
    gb = Basis(workload(name))
    plain = gb.scf(precision=FSIM_MIXED, tau=1e-10)
    dw = gb.scf(precision=FSIM_MIXED, tau=1e-10, dw_screen=True)
    assert plain["converged"] and dw["converged"]
    assert abs(dw["e_total"] - plain["e_total"]) < 1e-8
    per_build_plain = plain["quartets"] / (plain["fp64_builds"] + plain["mixed_builds"])
    per_build_dw = dw["quartets"] / (dw["fp64_builds"] + dw["mixed_builds"])
    assert per_build_dw < per_build_plain
    if name == "water8":
        gold = os.path.join(os.path.dirname(__file__), "golden", "water8_scf_oracle.json")
        with open(gold) as f:
            assert abs(dw["e_total"] - json.load(f)["e_total"]) < 1e-8
