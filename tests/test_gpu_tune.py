"""Autotuner: the table round-trips through a file and launch shapes never change results."""
import json

import numpy as np
import pytest

from paper_1812_07122_gb300 import blfls, synth

from gpu_util import smooth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def h():
    import __graft_entry__
    __graft_entry__.build()
    handle = blfls.blfls_create(0)
    yield handle
    blfls.blfls_destroy(handle)


def test_autotune_writes_a_table_that_create_reads(h, tmp_path):
    path = str(tmp_path / "tune.json")
    blfls.blfls_autotune(h, 256, 320, 1, 5, blfls.BLFLS_FP32, path)
    table = json.load(open(path))
    assert any(e["radius"] == 5 and e["prec"] == 0 for e in table["k1_tile_h"])
    assert table["k3_col_block"]
    h2 = blfls.blfls_create(0, 0, path)
    try:
        f = synth.sinusoid_disc_image(256, 320, 1, 20, seed=9)
        assert np.array_equal(smooth(h2, f, 30.0, 2.5, 0.1, 5), smooth(h, f, 30.0, 2.5, 0.1, 5))
    finally:
        blfls.blfls_destroy(h2)


@pytest.mark.parametrize("tile_h,col_block", [(8, 1), (16, 2), (64, 16)])
def test_every_launch_shape_gives_identical_results(h, tmp_path, tile_h, col_block):
    path = tmp_path / "t.json"
    path.write_text(json.dumps({"blfls_tune_table": 1,
                                "k1_tile_h": [{"radius": 5, "prec": 0, "tile_h": tile_h},
                                              {"radius": 10, "prec": 1, "tile_h": tile_h}],
                                "k3_col_block": [{"log2_len": 8, "col_block": col_block},
                                                 {"log2_len": 7, "col_block": col_block}]}))
    h2 = blfls.blfls_create(0, 0, str(path))
    try:
        for (H, W, C, r, prec) in [(200, 256, 2, 5, 0), (120, 100, 1, 10, 1)]:
            f = synth.sinusoid_disc_image(H, W, C, 10, seed=H)
            a = smooth(h2, f, 25.0, r / 2, 0.1, r, prec=prec)
            b = smooth(h, f, 25.0, r / 2, 0.1, r, prec=prec)
            assert np.array_equal(a, b), (tile_h, col_block, H, W)
    finally:
        blfls.blfls_destroy(h2)
