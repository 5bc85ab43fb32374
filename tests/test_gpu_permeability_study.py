"""Resolved vs homogenized permeability of a periodic sphere array on the GPU (the comparison
of the homogenized field with the pore-scale problem it stands in for)."""
import json

import pytest

from paper_2310_14746_gb300.workloads import permeability_pair

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2310_14746_gb300 import build
    build.build()


def test_resolved_vs_homogenized_vs_hasimoto():
    """One sphere per 32^3 periodic cell, r/P in {0.1, 0.2, 0.3}, tau = 0.8, FP32, run to
    max|du| < 1e-6 max|u| per 100 steps. The resolved (bounce-back) solve reproduces the
    dilute-array drag law within 5 %; the homogenized field of the same sphere (smoothed
    over 2 cells) gives a permeability of the same size (within 15 %: the smoothed edge and
    the finite penalisation move the effective surface by a fraction of a cell); both fall
    with the sphere size."""
    rows = [permeability_pair(32, r) for r in (0.1, 0.2, 0.3)]
    for row in rows:
        print(json.dumps(row))
    for row in rows:
        assert row["residual_resolved"] < 1e-6 and row["residual_homogenized"] < 1e-6
        assert abs(row["k_resolved"] - row["k_hasimoto"]) / row["k_hasimoto"] < 0.05
        assert abs(row["k_homogenized"] - row["k_resolved"]) / row["k_resolved"] < 0.15
    assert rows[0]["k_resolved"] > rows[1]["k_resolved"] > rows[2]["k_resolved"]
    assert rows[0]["k_homogenized"] > rows[1]["k_homogenized"] > rows[2]["k_homogenized"]
