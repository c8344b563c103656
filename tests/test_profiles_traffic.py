"""The DRAM traffic that bench.py reports in its roofline entry comes from the
ncu summaries under profiles/: every entry of its table must equal the
summary's dram__bytes_read.sum + dram__bytes_write.sum of the same launch
(CPU only; reads committed text)."""
import os
import re
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402

_UNIT = {"byte": 1.0, "Kbyte": 1e3, "Mbyte": 1e6, "Gbyte": 1e9}


def _dram_bytes(path, metric):
    text = open(os.path.join(ROOT, path)).read()
    m = re.search(r"`%s`\)\s*\|\s*([0-9.]+)\s*(byte|Kbyte|Mbyte|Gbyte)\s*\|" % re.escape(metric), text)
    assert m, "%s: no %s row" % (path, metric)
    return float(m.group(1)) * _UNIT[m.group(2)]


@pytest.mark.parametrize("name", sorted(bench.NCU_TRAFFIC))
def test_traffic_table_matches_the_profile(name):
    t = bench.NCU_TRAFFIC[name]
    total = _dram_bytes(t["profile"], "dram__bytes_read.sum") + _dram_bytes(t["profile"], "dram__bytes_write.sum")
    assert abs(t["bytes"] - total) <= 1e-4 * total, (name, t["bytes"], total)
    # the capture's lattice is the one the table scales from
    dims = re.search(r"(\d+)x(\d+)x(\d+)x(\d+)_ntv(\d+)", t["profile"])
    assert dims and int(dims.group(5)) == t["ntv"]
    assert t["sites"] == int(dims.group(1)) * int(dims.group(2)) * int(dims.group(3)) * int(dims.group(4))
