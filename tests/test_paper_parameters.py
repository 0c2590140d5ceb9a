"""The defaults of the oracle's parameter builder are the values the paper
prints (tests/golden/paper_parameters.json, each entry cited)."""
import json
import math
import os

import numpy as np

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_parameters.json")


def test_oracle_defaults_are_the_papers(orc):
    g = json.load(open(GOLDEN))
    p = orc.make_params()
    assert p.n_th == g["N_th"]["value"]
    assert p.cos_step == np.float32(math.cos(math.radians(g["theta_th_deg"]["value"])))
    assert p.cos_ccl == np.float32(math.cos(math.radians(g["theta_th_deg"]["value"])))
    assert p.n_hyp == g["ransac_iterations"]["value"]
    assert p.eps == np.float32(g["ransac_eps_m"]["value"])
    assert p.d_th2 == np.float32(g["d_th_m"]["value"] ** 2)
