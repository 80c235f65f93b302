"""The numbers the paper prints that this implementation adopts (stored in
tests/golden/paper_values.json with their citations), and Table 1's
post-activation centrality of exactly 0 reproduced by the oracle."""
import json
import os

import numpy as np

from paper_2508_10743_gb300 import configs

GOLDEN = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))


def test_defaults_follow_the_paper():
    d = configs.DarcConfig()
    assert d.n_squarings == GOLDEN["squarings"]["value"]
    assert d.lr == GOLDEN["adam_lr"]["value"]
    assert d.atlas_epochs == GOLDEN["K3_atlas_epochs"]["value"]
    assert configs.WORKLOADS["brain"].config.atlas_batch == GOLDEN["batch_oasis"]["value"]
    assert configs.WORKLOADS["cardiac"].config.atlas_batch == GOLDEN["batch_cardiac"]["value"]


def test_table1_centrality_after_activation_is_zero(ora):
    rng = np.random.default_rng(0)
    v = rng.normal(size=(6, 3, 5, 6, 7))
    ora.centrality(v)
    assert round(ora.centrality_metric(v) * 1e3, 1) == GOLDEN["centrality_after_activation_x1e3"]["value"]
