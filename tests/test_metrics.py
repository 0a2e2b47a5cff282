"""The flop and byte model used by the benchmark reproduces Table I of the paper
(tests/golden/table1.txt, Sec. II B 3)."""
import os

from paper_1712_01505_gb300 import metrics

HERE = os.path.dirname(os.path.abspath(__file__))


def _table1():
    rows = {}
    for line in open(os.path.join(HERE, "golden", "table1.txt")):
        if line.startswith("#") or not line.strip():
            continue
        name, flop, nbytes, ratio = line.split()
        rows[name] = (int(flop), int(nbytes), float(ratio))
    return rows


def test_wilson_row():
    flop, nbytes, ratio = _table1()["wilson"]
    assert metrics.table1_wilson("f32") == (flop, nbytes)
    assert round(nbytes / flop, 2) == ratio
    assert metrics.HOP_FLOP_SITE == 1320


def test_domain_wall_row_ns8():
    flop, nbytes, ratio = _table1()["domain_wall"]
    assert metrics.table1_domain_wall(8, "f32") == (flop, nbytes)
    assert round(nbytes / flop, 2) == ratio


def test_roofline_bytes():
    assert metrics.hop_compulsory_bytes("f32", 12) == 576
    assert metrics.hop_compulsory_bytes("f32", 18) == 768
    assert metrics.hop_compulsory_bytes("f64", 18) == 1536
    assert metrics.hop_compulsory_bytes("f16", 12) == 296
    assert metrics.hop_compulsory_bytes("f32", 12, slices=16) == 216
