"""The command-line tool on the GPU: a map shot in bands, interrupted and resumed from its
checkpoint file, equals the one-shot map bit for bit (exact FP32 path and far field)."""
import json

import numpy as np
import pytest

from paper_1005_5198_gb300 import cli

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("over", [[], ["precision=far32", "far_block=2"]], ids=["fp32c", "far32"])
def test_interrupted_banded_run_resumes_to_the_one_shot_map(tmp_path, over):
    one, banded, ckpt = tmp_path / "one.npy", tmp_path / "banded.npy", str(tmp_path / "map.ckpt.npz")
    assert cli.main(["shoot", "--config", "small", *sum((["--set", o] for o in over), []), "--out", str(one),
                     "--stats", str(tmp_path / "one.json")]) == 0
    args = ["shoot", "--config", "small", *sum((["--set", o] for o in over), []), "--out", str(banded),
            "--parts", "5", "--checkpoint", ckpt]
    assert cli.main(args + ["--max-parts-this-run", "2"]) == cli.EXIT_INTERRUPTED      # the first run stops
    assert not banded.exists()
    assert cli.main(args + ["--max-parts-this-run", "1"]) == cli.EXIT_INTERRUPTED      # a second short run
    assert cli.main(args) == 0                                                           # the rest
    a, b = np.load(one), np.load(banded)
    assert a.dtype == np.uint32 and a.shape == (128, 128)
    np.testing.assert_array_equal(a, b)
    st = json.loads((tmp_path / "one.json").read_text())
    assert st["rays_shot"] == st["geometry"]["nx"] * st["geometry"]["ny"] and st["rays_in"] == int(a.sum())


def test_checkpoint_of_another_config_is_refused(tmp_path):
    ckpt = str(tmp_path / "c.npz")
    base = ["shoot", "--config", "small", "--out", str(tmp_path / "m.npy"), "--parts", "3", "--checkpoint", ckpt]
    assert cli.main(base + ["--max-parts-this-run", "1"]) == cli.EXIT_INTERRUPTED
    with pytest.raises(SystemExit):
        cli.main(base + ["--set", "sigma=0.45"])


def test_image_and_lightcurve(tmp_path):
    img = tmp_path / "m.png"
    assert cli.main(["shoot", "--config", "small", "--out", str(tmp_path / "m.npy"), "--image", str(img)]) == 0
    assert img.read_bytes()[:8] == b"\x89PNG\r\n\x1a\n"
    lc_path = tmp_path / "lc.npy"
    assert cli.main(["lightcurve", "--config", "small", "--profile", "gaussian", "--size", "0.05",
                     "--start=-1.5,0", "--end=1.5,0.2", "--points", "300", "--out", str(lc_path)]) == 0
    lc = np.load(lc_path)
    assert lc.shape == (300,) and np.isfinite(lc).all() and (lc > 0).all()
