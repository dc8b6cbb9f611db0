"""The configuration constants against the values the paper prints: Table 1's variances
and weights (tests/golden/table1_variances_weights.txt, transcribed from the table), as
the oracle and the library's binding build their default configurations, and the level
that SSGI leaves out."""
import math
import os

import pytest

import oracle as orc

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "table1_variances_weights.txt")


def table1():
    rows = {}
    for line in open(GOLDEN):
        line = line.split("#", 1)[0].strip()
        if not line:
            continue
        effect, i, s2, w = line.split()
        rows.setdefault(effect, {})[int(i)] = None if s2 == "--" else (float(s2), float(w))
    return rows


def check(cfg, rows):
    for i in range(4):                       # level i is the paper's sub-image i + 1
        row = rows[i + 1]
        if row is None:
            assert cfg["enabled"][i] == 0
        else:
            assert cfg["enabled"][i] == 1
            assert cfg["sigma2"][i] == pytest.approx(row[0], abs=0)
            assert cfg["weight"][i] == pytest.approx(row[1], abs=0)


@pytest.mark.parametrize("effect", ["ssao", "ssm", "ssgi"])
def test_oracle_defaults_follow_table1(effect):
    check(orc.default_config(effect, 4), table1()[effect])


@pytest.fixture(scope="module")
def mrr():
    import __graft_entry__
    __graft_entry__.build()
    import paper_1906_04576_gb300 as m
    return m


@pytest.mark.parametrize("effect", ["ssao", "ssm", "ssgi"])
def test_library_defaults_follow_table1(mrr, effect):
    check(mrr.default_config(effect, 4, 64, 64), table1()[effect])


def test_blur_radii_of_table1_variances():
    """The truncation reading R = ceil(3 sigma) turns Table 1's variances into radii 3, 5
    and 6 -- the three patterns the mask kernels are compiled for."""
    radii = sorted({math.ceil(3 * math.sqrt(r[0])) for rows in table1().values()
                    for r in rows.values() if r and r[0] > 0})
    assert radii == [3, 5, 6]
    assert [len(orc.gauss_weights(s)) for s in (0.924, 1.848, 3.696)] == [7, 11, 13]
