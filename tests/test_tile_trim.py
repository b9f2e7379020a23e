"""The binning's column cuts never drop a tile holding a pixel that passes the
blend's alpha test (host build of the kernel's own header; no GPU), and they
do remove a good share of the rectangles' tiles."""
import shutil
import subprocess
from pathlib import Path

import pytest

ROOT = Path(__file__).resolve().parents[1]


@pytest.fixture(scope="module")
def checker(tmp_path_factory):
    cxx = shutil.which("g++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    exe = tmp_path_factory.mktemp("trim") / "tile_trim_check"
    subprocess.run([cxx, "-O2", "-std=c++17", "-ffp-contract=off", "-I", str(ROOT / "paper_2503_22159_gb300" / "csrc"),
                    str(ROOT / "tests" / "tile_trim_check.cpp"), "-o", str(exe)], check=True)
    return exe


def test_column_cuts_are_conservative(checker):
    r = subprocess.run([str(checker), "3000"], capture_output=True, text=True)
    assert r.returncode == 0, r.stdout + r.stderr
    rows = [list(map(int, line.split())) for line in r.stdout.strip().splitlines()]
    assert [row[0] for row in rows] == [8, 16, 32]
    for ts, rect, kept, needed, failures in rows:
        assert failures == 0
        assert needed <= kept <= rect
    # 32-px tiles: the cuts remove a sizeable share of the rectangles' tiles
    ts, rect, kept, needed, _ = rows[2]
    assert kept < 0.8 * rect
