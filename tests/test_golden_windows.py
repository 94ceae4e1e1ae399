"""Window counts against the paper's printed example (tests/golden/window_counts.txt): one window
per starting sample of a 4096 s, 4096 Hz segment gives 4096 x 4096 - 4096 + 1 windows, and three
segments about 50M.  Checked for the oracle and for the library's host-side count (no GPU call)."""
import os

import oracle

HERE = os.path.dirname(os.path.abspath(__file__))


def _rows():
    rows = []
    with open(os.path.join(HERE, "golden", "window_counts.txt")) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append(tuple(int(v) for v in line.split()))
    return rows


def test_oracle_window_count_matches_paper():
    rows = _rows()
    assert rows
    for n, w, s, nw in rows:
        assert oracle.n_windows(n, w, s) == nw
    n, w, s, nw = rows[0]
    assert 49.5e6 < 3 * nw < 50.5e6          # "about 50M" over three segments


def test_library_window_count_matches_paper():
    import paper_2201_11133_gb300 as gwe
    for n, w, s, nw in _rows():
        assert gwe.gwe_n_windows(n, w, s) == nw
