"""The bit-rate / topology-error trade-off (Section III-B, Table II) from the
CUDA path against the same quantities from the oracle: stream size, FN / FP /
FT per critical-point type, and the largest error over the bound."""
import numpy as np
import pytest
import torch

import oracle
from paper_2602_17552_gb300 import codec, synth

pytestmark = pytest.mark.gpu

FIELDS = [
    ("climate_300x517", lambda: synth.climate_2d(300, 517, seed=2).numpy()),
    ("turb_40", lambda: synth.turbulence_3d(40, seed=3).numpy()),
]


@pytest.mark.parametrize("name,make", FIELDS, ids=[f[0] for f in FIELDS])
def test_tradeoff_matches_oracle(name, make):
    a = make()
    f = torch.from_numpy(a).cuda()
    lab_a = oracle.critical_points(a)
    for eb in (1e-3, 1e-4, 1e-5):
        for no_topo in (False, True):
            row = codec.tradeoff(f, eb, "rel", no_topo=no_topo)
            obuf = oracle.compress(a, eb, rel=True, no_topo=no_topo)
            oout = oracle.decompress(obuf, a.shape)
            e = oracle.topo_errors(lab_a, oracle.critical_points(oout))
            assert row["bytes"] == len(obuf), (eb, no_topo)
            assert [row["fn"], row["fp"], row["ft"]] == e.tolist(), (eb, no_topo)
            err = float(np.abs(oout.astype(np.float64) - a.astype(np.float64)).max())
            assert row["max_err_over_eps"] == pytest.approx(err / oracle.header(obuf)["eps"], rel=1e-12)
            # the bound: within eps without the topology stage, within 2 eps with it
            assert row["max_err_over_eps"] <= (2.0 if not no_topo else 1.0)
