"""The persistent DTW tile cache (environment variable TCDTW_TUNE_CACHE).

tcdtw_build times the compiled band tiles on the candidates and keeps the fastest
(tile, G) per (L, D, W) for the life of the process; with TCDTW_TUNE_CACHE naming a
file, choices are read from it on first use and every new tuning is appended.  Lines
of another device or of another build's tile table (its FNV-1a signature over the
compiled (R, maxD) list) are ignored.  The file is read once per process, so each case
runs in a fresh interpreter.
"""
import json
import os
import subprocess
import sys

import pytest
import torch

pytestmark = pytest.mark.gpu

tc = pytest.importorskip("paper_2101_07731_gb300")
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

_BUILD = r"""
import json, sys
sys.path.insert(0, {root!r})
import torch
import paper_2101_07731_gb300 as tc
import synth
spec = synth.SeriesSpec("random_walk", {L}, {D}, 5)
cand = torch.from_numpy(synth.generate(spec, synth.ROLE_CAND, 600)).cuda()
x = tc.Index(cand, {W}, 8)
print(json.dumps(x.info()))
x.close()
"""


def _build_info(L, D, W, cache):
    env = dict(os.environ)
    env.pop("TCDTW_TUNE_CACHE", None)
    if cache is not None:
        env["TCDTW_TUNE_CACHE"] = str(cache)
    out = subprocess.run([sys.executable, "-c", _BUILD.format(root=ROOT, L=L, D=D, W=W)], env=env,
                         capture_output=True, text=True, timeout=300)
    assert out.returncode == 0, out.stderr[-2000:]
    return json.loads(out.stdout.strip().splitlines()[-1])


def _tiles():
    lib = tc._load()
    import ctypes as C
    tiles = []
    for t in range(lib.tcdtw_tile_count()):
        r, dm = C.c_int32(), C.c_int32()
        assert lib.tcdtw_tile_info(t, None, C.byref(r), C.byref(dm)) == 0
        tiles.append((r.value, dm.value))
    return tiles


def _signature(tiles):
    h = 2166136261
    for r, dm in tiles:
        h = ((h ^ r) * 16777619) & 0xFFFFFFFF
        h = ((h ^ dm) * 16777619) & 0xFFFFFFFF
    return h


def test_tune_cache_is_read_validated_and_appended(tmp_path):
    L, D, W = 64, 3, 6
    tiles = _tiles()
    tag = torch.cuda.get_device_name(0).replace(" ", "_").replace("\t", "_")
    sig = _signature(tiles)
    tuned = _build_info(L, D, W, None)          # the tuner's own choice, no cache
    dm = tiles[tuned["tile"]][1]
    # another valid choice of the same width bucket: a (tile, G) the tuner did not pick
    alt = [(t, g) for t, (r, d) in enumerate(tiles) if d == dm for g in (4, 8, 16, 32)
           if g * (r + 1) >= 2 * W + r and (t, g) != (tuned["tile"], tuned["G"])]
    assert alt
    t1, g1 = alt[0]
    f = tmp_path / "tune.txt"
    f.write_text(f"tcdtw-tune {sig ^ 1:x} {tag} {L} {D} {W} {alt[-1][0]} {alt[-1][1]}\n"   # foreign build
                 f"tcdtw-tune {sig:x} {tag} {L} {D} {W} {t1} {g1}\n")
    got = _build_info(L, D, W, f)
    assert (got["tile"], got["G"]) == (t1, g1), (got, t1, g1)
    # a shape not in the file is tuned and appended
    _build_info(80, D, 5, f)
    lines = f.read_text().splitlines()
    new = [ln.split() for ln in lines if ln.split()[3:6] == ["80", str(D), "5"]]
    assert len(new) == 1 and new[0][1] == f"{sig:x}" and new[0][2] == tag
