"""The oracle's codings against the byte column that Table I prints (fixture
`tests/golden/table1_sh_bytes.txt`, every row of the table with its block setup, Sec. V-B).

Setups A and B: the bytes of the coded blocks per primitive equal the printed value, in both
orders. Setup D: the table prints 8.5 / 9 / 17 where the blocks (8 B per BC1 block, 16 B per BC7
block, 16 blocks for 16 primitives) come to 8 / 8.5 / 16. All six D rows equal the block bytes
plus one more block per group of 16 primitives in the format of the group's other blocks
(17 x 8 / 16, (16 + 16 x 8) / 16, 17 x 16 / 16; a uniform 17/16 factor would give 9.03 for the
middle row), which this file checks; the codec's rate is the block bytes (the reading of those
rows). The 8-bit row equals the 48 quantised texels of one primitive; the
FP32 row prints 196 B where 48 four-byte floats are 192 B (the colour input here is 192 B).
"""
import os

import numpy as np

from paper_2607_14513_gb300 import synthetic as S

HERE = os.path.dirname(os.path.abspath(__file__))
LAYOUT = {"D": 0, "A": 1, "B": 2}


def _rows():
    rows = []
    with open(os.path.join(HERE, "golden", "table1_sh_bytes.txt")) as f:
        for line in f:
            line = line.split("#", 1)[0].split()
            if line:
                setup, j, order, printed = line
                rows.append((setup, None if j == "-" else int(j), order, float(printed)))
    return rows


def test_fixture_holds_every_row_of_the_table():
    rows = _rows()
    assert len(rows) == 12
    assert [r[0] for r in rows] == ["fp32", "q8", "A", "A", "B", "B", "D", "D", "D", "D", "D", "D"]


def test_codings_match_the_printed_bytes(O):
    sc = S.make_scene(**S.TINY)
    n = 512
    sh = sc.sh[:n]
    scales = O.scales(sh)
    q = O.quantise(sh, scales)
    orders = {"original": np.arange(n, dtype=np.int32), "-": np.arange(n, dtype=np.int32),
              "sorted": np.asarray(O.plan(sc.pos[:n], q, 256, 1), np.int32)}
    for setup, j, order, printed in _rows():
        if setup == "fp32":
            assert sh.dtype == np.float32 and sh[0].nbytes == 192 and printed == 196
            continue
        if setup == "q8":
            assert q.dtype == np.uint8 and q[0].nbytes == printed
            continue
        perm = orders[order]
        r = O.encode_layout(q, perm, scales, LAYOUT[setup], j)
        got = r["table"].total_bytes / n
        assert got == 8.0 * (16 - j) / 16 + 16.0 * j / 16, (setup, j)    # the block arithmetic
        if setup in ("A", "B"):
            assert got == printed, (setup, j, order)
        else:
            # Setup D rows: one more block per group of 16, in the format of the group's last block
            extra = (16.0 if j == 16 else 8.0) / 16
            assert printed == got + extra, (setup, j, order)
