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
    rows = [permeability_pair(32, r) for r in (0.1, 0.2, 0.3)]
    for row in rows:
        print(json.dumps(row))
        # the resolved solve reproduces the dilute-array drag law
        assert abs(row["k_resolved"] - row["k_hasimoto"]) / row["k_hasimoto"] < 0.05
        # the homogenized (penalised, smoothed) sphere is more permeable than the no-slip one
        assert row["k_homogenized"] > row["k_resolved"]
    # permeability falls with the sphere size in both descriptions
    assert rows[0]["k_resolved"] > rows[1]["k_resolved"] > rows[2]["k_resolved"]
    assert rows[0]["k_homogenized"] > rows[1]["k_homogenized"] > rows[2]["k_homogenized"]
