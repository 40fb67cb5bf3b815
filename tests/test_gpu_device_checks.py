"""The debug build's device range checks (GPU).

The library is built once more with -DBLFLS_DEVICE_CHECKS (its own directory), and a child
process loaded with that build runs the main paths: the plain smoother in every precision at
ragged sizes, the runtime-window and per-pixel bilateral kernels, the 4K channel on the
compile-time FFT plans, a Bluestein size, the batched form, the grid, NC-LS, normalised and
guided smoothing.  Every check must pass (the word blfls_device_checks returns stays 0), and
the results must be those of the release build: the checks only skip accesses that would leave
their buffers, so FP32 and BF16W results are the same bits; FP16W may differ by an output ulp
(the compiler rounds subnormal FP16 weights per kernel build).
"""
import os
import subprocess
import sys

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

WORKLOAD = r'''
import sys
import numpy as np
import torch
sys.path.insert(0, ROOT)
from paper_1812_07122_gb300 import blfls, synth

dev = torch.device("cuda:0")
s = torch.cuda.current_stream(dev)
h = blfls.blfls_create(0)
res = {}

def run(name, fn, f):
    x = torch.from_numpy(np.ascontiguousarray(f, dtype=np.float32)).to(dev)
    out = torch.empty_like(x)
    fn(x, out)
    torch.cuda.synchronize(dev)
    res[name] = out.cpu().numpy()

f3 = synth.sinusoid_disc_image(57, 71, 3, n_disc=5, noise=0.03, seed=7)
for prec in (0, 1, 2):
    run(f"smooth_{prec}", lambda x, o, p=prec: blfls.blfls_smooth(h, x, o, 57, 71, 3, 30.0, 4.0,
        0.08, 8, 2, p, s), f3)
f1 = synth.sinusoid_disc_image(110, 123, 1, n_disc=5, noise=0.03, seed=8)
for r in (20, 50):
    run(f"radius_{r}", lambda x, o, r=r: blfls.blfls_smooth(h, x, o, 110, 123, 1, 20.0, r / 2,
        0.1, r, 1, 0, s), f1)
f4k = synth.image_4k_rgb()[:1]
run("4k", lambda x, o: blfls.blfls_smooth(h, x, o, 2160, 3840, 1, 30.0, 5.0, 0.08, 10, 1, 0, s),
    f4k)
fb = synth.sinusoid_disc_image(211, 97, 1, n_disc=5, noise=0.03, seed=9)
run("bluestein", lambda x, o: blfls.blfls_smooth(h, x, o, 211, 97, 1, 20.0, 2.5, 0.1, 5, 1, 1,
    s), fb)
run("grid", lambda x, o: blfls.blfls_smooth_grid(h, x, o, 57, 71, 3, 30.0, 3.0, 0.08, 1, s), f3)
run("nc", lambda x, o: blfls.blfls_smooth_nc(h, x, o, 57, 71, 3, 30.0, 5.0, 0.05, 1, 3, s), f3)
run("normalized", lambda x, o: blfls.blfls_smooth_normalized(h, x, o, 57, 71, 3, 30.0, 4.0,
    0.08, 8, 1, 0, s), f3)
run("guided", lambda x, o: blfls.blfls_smooth_guided(h, x, x, o, 57, 71, 3, 3, 30.0, 4.0, 0.08,
    8, 1, 0, s), f3)
xs = [torch.from_numpy(synth.sinusoid_disc_image(H, W, C, n_disc=4, seed=H + W)).to(dev)
      for H, W, C in ((64, 80, 1), (97, 61, 3), (128, 257, 1))]
outs = [torch.empty_like(x) for x in xs]
jobs = [blfls.make_job(x, o, x.shape[1], x.shape[2], x.shape[0], 20.0, 2.5, 0.1, 5)
        for x, o in zip(xs, outs)]
blfls.blfls_smooth_batch(h, jobs, s)
torch.cuda.synchronize(dev)
for i, o in enumerate(outs):
    res[f"batch_{i}"] = o.cpu().numpy()
res["word"] = np.array([blfls.blfls_device_checks(0)], dtype=np.int64)
blfls.blfls_destroy(h)
np.savez(OUT, **res)
'''


def _run(lib, out):
    env = dict(os.environ)
    if lib:
        env["BLFLS_LIBRARY"] = lib
    else:
        env.pop("BLFLS_LIBRARY", None)
    code = f"ROOT = {ROOT!r}\nOUT = {str(out)!r}\n" + WORKLOAD
    p = subprocess.run([sys.executable, "-c", code], env=env, cwd=ROOT, capture_output=True,
                       text=True, timeout=900)
    assert p.returncode == 0, p.stdout[-2000:] + p.stderr[-2000:]
    return np.load(out)


def test_debug_build_checks_pass_and_match_the_release_build(tmp_path):
    import __graft_entry__
    from paper_1812_07122_gb300 import build
    __graft_entry__.build()
    debug_lib = build.build(debug=True)
    rel = _run(None, tmp_path / "release.npz")
    dbg = _run(debug_lib, tmp_path / "debug.npz")
    assert int(rel["word"][0]) == 0                  # release: the checks compile away
    assert int(dbg["word"][0]) == 0, f"device range checks failed: {int(dbg['word'][0]):#x}"
    for name in rel.files:
        if name == "word":
            continue
        if name in ("smooth_1", "bluestein"):        # FP16W
            assert float(np.max(np.abs(rel[name] - dbg[name]))) <= 1e-6, name
        else:
            np.testing.assert_array_equal(rel[name], dbg[name], err_msg=name)
