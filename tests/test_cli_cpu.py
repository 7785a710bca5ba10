"""The command-line tool's host side: shipped configs, overrides, geometry, band plans, PNG output."""
import json

import numpy as np
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


def test_png_writer_round_trip(tmp_path):
    import struct
    import zlib
    img = (np.arange(6 * 5, dtype=np.uint32).reshape(6, 5) * 7 % 256).astype(np.uint8)
    path = tmp_path / "m.png"
    cli.write_png(str(path), img)
    data = path.read_bytes()
    assert data[:8] == b"\x89PNG\r\n\x1a\n"
    pos, chunks = 8, {}
    while pos < len(data):
        (n,) = struct.unpack(">I", data[pos:pos + 4])
        tag, body = data[pos + 4:pos + 8], data[pos + 8:pos + 8 + n]
        assert struct.unpack(">I", data[pos + 8 + n:pos + 12 + n])[0] == zlib.crc32(tag + body) & 0xFFFFFFFF
        chunks[tag] = chunks.get(tag, b"") + body
        pos += 12 + n
    w, h, depth, colour = struct.unpack(">IIBB", chunks[b"IHDR"][:10])
    assert (w, h, depth, colour) == (5, 6, 8, 0)
    raw = zlib.decompress(chunks[b"IDAT"])
    rows = [raw[r * 6 + 1:(r + 1) * 6] for r in range(6)]
    assert np.array_equal(np.frombuffer(b"".join(rows), dtype=np.uint8).reshape(6, 5), img)


def test_delta_m_image_orientation_and_scale():
    counts = np.zeros((4, 4), dtype=np.uint32)
    counts[0, 0] = 100          # row 0 (lowest y2) is the image's bottom row
    counts[3, 3] = 1
    img = cli.delta_m_image(counts, 10.0)
    assert img[3, 0] == 255 and img[0, 3] == 1           # most magnified bright, least dim
    assert (img == 0).sum() == 14                          # no ray: black
