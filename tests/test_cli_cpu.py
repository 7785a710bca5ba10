"""The command-line tool's host side: shipped configs, overrides, geometry, band plans."""
import json

import pytest

import paper_1005_5198_gb300 as mm
from paper_1005_5198_gb300 import cli


def test_shipped_configs_load_and_give_the_paper_geometry():
    assert set(cli.shipped_configs()) >= {"small", "fig1", "sigma08"}
    g = mm.mm_geometry_of(cli.to_params(cli.load_config("fig1")))
    assert (g["nx"], g["ny"], g["nstar"]) == (114487, 114487, 558)          # Fig. 1: N* = 558 (Sect. 3.2.1)
    p = cli.to_params(cli.load_config("sigma08"))
    assert p.precision == mm.MM_FAR32 and p.nstar == 25000 and p.far_order == 10


def test_overrides_and_errors(tmp_path):
    cfg = cli.load_config("small", ["npix_side=64", "precision=fp64"])
    p = cli.to_params(cfg)
    assert p.npix_side == 64 and p.precision == mm.MM_FP64
    bad = tmp_path / "bad.json"
    bad.write_text(json.dumps({"sigma": 0.4, "gama": 0.1}))
    with pytest.raises(ValueError):
        cli.load_config(str(bad))
    with pytest.raises(ValueError):
        cli.load_config("small", ["precision=fp16"])
    with pytest.raises(ValueError):
        cli.load_config("no-such-config")


def test_geometry_command_prints_the_library_geometry(capsys):
    assert cli.main(["geometry", "--config", "small"]) == 0
    out = json.loads(capsys.readouterr().out)
    assert out == mm.mm_geometry_of(cli.to_params(cli.load_config("small")))


@pytest.mark.parametrize("ny,parts,align", [(3200, 4, 32), (114487, 8, 32), (100, 8, 32), (68693, 5, 256), (31, 3, 32)])
def test_band_plan_covers_the_rows_once_on_the_tile_grid(ny, parts, align):
    plan = cli.band_plan(ny, parts, align)
    assert plan[0] == 0 and plan[-1] == ny and len(plan) - 1 <= parts
    assert all(a < b for a, b in zip(plan, plan[1:]))
    assert all(j % align == 0 for j in plan[:-1])
